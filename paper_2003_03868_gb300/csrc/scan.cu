// Prefix sums and a deterministic FP64 sum, used by the stack builder and the
// filter compaction.  Three-phase scan: every CTA scans one tile and records its
// total, the tile totals are scanned (recursively), and the tile offsets are
// added back.
#include "common.cuh"

namespace dbg {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kTile = kScanThreads * kScanItems;

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t* warp_tot, int64_t& excl) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t t = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;   // inclusive over warps
    }
    __syncthreads();
    int64_t before = (warp > 0) ? warp_tot[warp - 1] : 0;
    excl = before + x - v;
    int64_t total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return total;
}

template <class T>
__global__ void k_scan_tiles(const T* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                             int64_t* __restrict__ tile_sums) {
    __shared__ int64_t warp_tot[32];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
    int64_t vals[kScanItems];
    int64_t local = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        vals[i] = (idx < n) ? (int64_t)in[idx] : 0;
        local += vals[i];
    }
    int64_t excl;
    int64_t total = block_exclusive_scan(local, warp_tot, excl);
    int64_t run = excl;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += vals[i];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void k_add_tile_offsets(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ tile_off) {
    const int64_t off = tile_off[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += blockDim.x) {
        int64_t idx = base + i;
        if (idx < n) out[idx] += off;
    }
}

__global__ void k_set_total(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ tile_scan,
                            int64_t ntiles) {
    out[n] = tile_scan[ntiles];
}

template <class T>
void scan_impl(const T* in, int64_t* out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        DBG_CK(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return;
    }
    const int64_t ntiles = ceil_div(n, kTile);
    DBuf<int64_t> sums;
    sums.alloc(ntiles, s);
    k_scan_tiles<T><<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, out, n, sums.p);
    DBG_LAUNCH_CK();
    if (ntiles == 1) {
        // one tile: its total is the total
        k_set_total<<<1, 1, 0, s>>>(out, n, sums.p, 0);
        DBG_LAUNCH_CK();
        return;
    }
    DBuf<int64_t> sums_scan;
    sums_scan.alloc(ntiles + 1, s);
    scan_impl<int64_t>(sums.p, sums_scan.p, ntiles, s);
    k_add_tile_offsets<<<(unsigned)ntiles, kScanThreads, 0, s>>>(out, n, sums_scan.p);
    DBG_LAUNCH_CK();
    k_set_total<<<1, 1, 0, s>>>(out, n, sums_scan.p, ntiles);
    DBG_LAUNCH_CK();
}

constexpr int kSumThreads = 256;
constexpr int kSumBlocks = 1024;
static_assert(kSumBlocks == kDetSumPartials, "det_sum_into partial count");

// Each CTA sums a fixed contiguous chunk (thread-strided, then a fixed tree).
__global__ void k_sum_partials(const double* __restrict__ v, int64_t n, double* __restrict__ part) {
    __shared__ double sh[kSumThreads];
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * chunk;
    const int64_t hi = min(n, lo + chunk);
    double s = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += v[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kSumThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_final(const double* __restrict__ part, int np, double* __restrict__ out) {
    __shared__ double sh[kSumBlocks];
    for (int i = threadIdx.x; i < kSumBlocks; i += blockDim.x) sh[i] = (i < np) ? part[i] : 0.0;
    __syncthreads();
    for (int w = kSumBlocks / 2; w > 0; w >>= 1) {
        for (int i = threadIdx.x; i < w; i += blockDim.x) sh[i] += sh[i + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

}  // namespace

void scan_exclusive(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) { scan_impl<int64_t>(in, out, n, s); }
void scan_exclusive(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) { scan_impl<int32_t>(in, out, n, s); }

void det_sum(const double* v, int64_t n, double* out, cudaStream_t s) {
    if (n <= 0) {
        DBG_CK(cudaMemsetAsync(out, 0, sizeof(double), s));
        return;
    }
    DBuf<double> part;
    part.alloc(kSumBlocks, s);
    k_sum_partials<<<kSumBlocks, kSumThreads, 0, s>>>(v, n, part.p);
    DBG_LAUNCH_CK();
    k_sum_final<<<1, 256, 0, s>>>(part.p, kSumBlocks, out);
    DBG_LAUNCH_CK();
}

void det_sum_into(const double* v, int64_t n, double* partials, double* out, cudaStream_t s) {
    if (n <= 0) {
        DBG_CK(cudaMemsetAsync(out, 0, sizeof(double), s));
        return;
    }
    k_sum_partials<<<kSumBlocks, kSumThreads, 0, s>>>(v, n, partials);
    DBG_LAUNCH_CK();
    k_sum_final<<<1, 256, 0, s>>>(partials, kSumBlocks, out);
    DBG_LAUNCH_CK();
}

}  // namespace dbg
