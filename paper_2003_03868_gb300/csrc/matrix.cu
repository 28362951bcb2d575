// Block-CSR matrices on the device: staging and finalize, copies, per-block
// norms, scale/shift, and the norm filter with its compaction.
//
// Layout (DBCSR section "DBCSR library": dense atom blocks in a blocked CSR
// format): row pointers rp[nblk+1], ascending block columns col[nnzb], the block
// row of each block row[nnzb], element offsets off[nnzb+1], and the blocks
// themselves row-major and packed in CSR order in data[nel] (FP64).
#include <algorithm>
#include <array>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "dbcsr_gb_bench.h"

namespace dbg {

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};
}  // namespace

cudaMemPool_t library_pool() {
    int dev = 0;
    DBG_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) fail(DBCSR_ECAPACITY, "library_pool: device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        DBG_CK(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = ~0ull;
        DBG_CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pools[dev] = pool;
    }
    return g_pools[dev];
}

int num_sms() {
    static std::atomic<int> cache[kMaxDevices] = {};
    int dev = 0;
    DBG_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) fail(DBCSR_ECAPACITY, "num_sms: device ordinal out of range");
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n <= 0) {
        DBG_CK(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        if (n <= 0) fail(DBCSR_ECUDA, "num_sms: no multiprocessors reported");
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

void trim_pool(uint64_t keep_bytes) {
    int dev = 0;
    DBG_CK(cudaGetDevice(&dev));
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (dev >= 0 && dev < kMaxDevices) pool = g_pools[dev];
    }
    if (!pool) return;
    DBG_CK(cudaDeviceSynchronize());
    DBG_CK(cudaMemPoolTrimTo(pool, (size_t)keep_bytes));
}

void pool_alloc(void** p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool = library_pool();
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        DBG_CK(cudaDeviceSynchronize());
        DBG_CK(cudaMemPoolTrimTo(pool, 0));
        e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? DBCSR_ENOMEM : DBCSR_ECUDA,
             std::string("device allocation of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
}

HostScalars::HostScalars() {
    DBG_CK(cudaMallocHost((void**)&i, kCap * sizeof(int64_t)));
    DBG_CK(cudaMallocHost((void**)&d, 64 * sizeof(double)));
}
HostScalars::~HostScalars() {
    if (i) cudaFreeHost(i);
    if (d) cudaFreeHost(d);
}
HostScalars& host_scalars() {
    static thread_local HostScalars hs;
    return hs;
}

int64_t read_i64(const int64_t* dev, cudaStream_t s) {
    HostScalars& hs = host_scalars();
    DBG_CK(cudaMemcpyAsync(hs.i, dev, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    DBG_CK(cudaStreamSynchronize(s));
    return hs.i[0];
}

void read_i64s(const int64_t* const* dev, int k, int64_t* out, cudaStream_t s, const int64_t* arr, int na,
               int64_t* arr_out) {
    HostScalars& hs = host_scalars();
    if (k + na > HostScalars::kCap) fail(DBCSR_ECAPACITY, "read_i64s: too many values");
    for (int j = 0; j < k; ++j) DBG_CK(cudaMemcpyAsync(hs.i + j, dev[j], sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (na > 0) DBG_CK(cudaMemcpyAsync(hs.i + k, arr, sizeof(int64_t) * na, cudaMemcpyDeviceToHost, s));
    DBG_CK(cudaStreamSynchronize(s));
    for (int j = 0; j < k; ++j) out[j] = hs.i[j];
    for (int j = 0; j < na; ++j) arr_out[j] = hs.i[k + j];
}

double read_f64(const double* dev, cudaStream_t s) {
    HostScalars& hs = host_scalars();
    DBG_CK(cudaMemcpyAsync(hs.d, dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    DBG_CK(cudaStreamSynchronize(s));
    return hs.d[0];
}

void check_unplanned(const dbcsr_matrix_* m, const char* where) {
    if (m && m->plans > 0)
        fail(DBCSR_ESTATE, std::string(where) + ": a multiply plan uses this matrix (destroy the plan first)");
}

void check_finalized(const dbcsr_matrix_* m) {
    if (!m) fail(DBCSR_EINVAL, "null matrix handle");
    if (!m->finalized) fail(DBCSR_ESTATE, "matrix is not finalized");
}

namespace {

// One warp per block: copies staged block b from the staging pool into CSR position.
__global__ void k_gather_blocks(int64_t nb, const int64_t* __restrict__ src_off, const double* __restrict__ pool,
                                const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                                const int32_t* __restrict__ bs, const int64_t* __restrict__ dst_off,
                                double* __restrict__ dst) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < nb; b += warps) {
        const double* src = pool + src_off[b];
        const int area = bs[row[b]] * bs[col[b]];
        double* d = dst + dst_off[b];
        for (int e = lane; e < area; e += 32) d[e] = src[e];
    }
}

// One warp per block: Frobenius norm (lane partials in element order, then a
// fixed xor-shuffle tree) and squared distance to the identity.
__global__ void k_block_norms(int64_t nb, const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                              const int32_t* __restrict__ bs, const int64_t* __restrict__ off,
                              const double* __restrict__ data, double* __restrict__ norms, double* __restrict__ dev2) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < nb; b += warps) {
        const int I = row[b], J = col[b];
        const int n = bs[J], area = bs[I] * n;
        const double* x = data + off[b];
        double s = 0.0, d = 0.0;
        if (I != J) {
            // off the diagonal the distance to 1 is the norm: one FMA chain (the FP64 rate,
            // not the memory, bounds this loop)
            for (int e = lane; e < area; e += 32) {
                const double v = x[e];
                s = fma(v, v, s);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            d = s;
        } else {
            // element e = i n + j of a square block is diagonal when e is a multiple of n + 1
            for (int e = lane; e < area; e += 32) {
                const double v = x[e];
                s = fma(v, v, s);
                const double w = (e % (n + 1) == 0) ? v - 1.0 : v;
                d = fma(w, w, d);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s += __shfl_xor_sync(0xffffffffu, s, o);
                d += __shfl_xor_sync(0xffffffffu, d, o);
            }
        }
        if (lane == 0) {
            if (norms) norms[b] = sqrt(s);
            if (dev2) dev2[b] = d;
        }
    }
}

__global__ void k_scale_shift(int64_t nb, const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                              const int32_t* __restrict__ bs, const int64_t* __restrict__ off, double* __restrict__ data,
                              double scale, double shift) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < nb; b += warps) {
        const int I = row[b], J = col[b];
        const int n = bs[J], area = bs[I] * n;
        double* x = data + off[b];
        if (I != J) {
            for (int e = lane; e < area; e += 32) x[e] = scale * x[e];
        } else {
            for (int e = lane; e < area; e += 32) {
                double v = scale * x[e];
                if (e % (n + 1) == 0) v += shift;     // the diagonal of a square block
                x[e] = v;
            }
        }
    }
}

// Flags every block row that lacks its diagonal block.
__global__ void k_missing_diag(int32_t nblk, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               int64_t* __restrict__ missing) {
    for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < nblk; I += gridDim.x * blockDim.x) {
        int64_t lo = rp[I], hi = rp[I + 1];
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (col[mid] < I) lo = mid + 1; else hi = mid;
        }
        if (!(lo < rp[I + 1] && col[lo] == I)) atomicAdd((unsigned long long*)missing, 1ull);
    }
}

__global__ void k_keep_norm(int64_t nb, const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                            const double* __restrict__ norms, double eps, int32_t* __restrict__ keep) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x)
        keep[b] = (row[b] == col[b] || norms[b] >= eps) ? 1 : 0;
}

// Compaction: kept block b goes to index newidx[b] with data at newoff[newidx[b]].
__global__ void k_compact_meta(int64_t nb, const int32_t* __restrict__ keep, const int64_t* __restrict__ newidx,
                               const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                               const int32_t* __restrict__ bs, const double* __restrict__ norms,
                               int32_t* __restrict__ nrow, int32_t* __restrict__ ncol, int64_t* __restrict__ narea,
                               double* __restrict__ nnorms) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[b]) continue;
        const int64_t k = newidx[b];
        nrow[k] = row[b];
        ncol[k] = col[b];
        narea[k] = (int64_t)bs[row[b]] * bs[col[b]];
        if (nnorms) nnorms[k] = norms[b];
    }
}

__global__ void k_compact_rp(int32_t nblk, const int64_t* __restrict__ rp, const int64_t* __restrict__ newidx,
                             int64_t* __restrict__ nrp) {
    for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I <= nblk; I += gridDim.x * blockDim.x)
        nrp[I] = newidx[rp[I]];
}

__global__ void k_compact_data(int64_t nb, const int32_t* __restrict__ keep, const int64_t* __restrict__ newidx,
                               const int64_t* __restrict__ off, const int64_t* __restrict__ noff,
                               const double* __restrict__ data, double* __restrict__ ndata) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < nb; b += warps) {
        if (!keep[b]) continue;
        const int64_t k = newidx[b];
        const int64_t area = off[b + 1] - off[b];
        const double* s = data + off[b];
        double* d = ndata + noff[k];
        for (int64_t e = lane; e < area; e += 32) d[e] = s[e];
    }
}

}  // namespace

void compute_block_norms(const dbcsr_matrix_* m, double* norms, double* dev2) {
    if (m->nnzb == 0) return;
    k_block_norms<<<grid_for(m->nnzb, 8), 256, 0, m->stream>>>(m->nnzb, m->row.p, m->col.p, m->bs.p, m->off.p,
                                                               m->data.p, norms, dev2);
    DBG_LAUNCH_CK();
}

void ensure_norms(dbcsr_matrix_* m) {
    if (m->norms_valid) return;
    m->norms.alloc(std::max<int64_t>(m->nnzb, 1), m->stream);
    compute_block_norms(m, m->norms.p, nullptr);
    m->norms_valid = true;
}

void copy_matrix(dbcsr_matrix_* dst, const dbcsr_matrix_* src) {
    check_unplanned(dst, "copy");
    check_finalized(src);
    if (dst == src) return;
    if (dst->h_bs != src->h_bs) fail(DBCSR_EINVAL, "copy: block sizes differ");
    cudaStream_t s = dst->stream;
    if (src->stream != s) DBG_CK(cudaStreamSynchronize(src->stream));
    dst->rp.alloc(src->nblk + 1, s);
    dst->col.alloc(std::max<int64_t>(src->nnzb, 1), s);
    dst->row.alloc(std::max<int64_t>(src->nnzb, 1), s);
    dst->off.alloc(src->nnzb + 1, s);
    dst->data.alloc(std::max<int64_t>(src->nel, 1), s);
    DBG_CK(cudaMemcpyAsync(dst->rp.p, src->rp.p, sizeof(int64_t) * (src->nblk + 1), cudaMemcpyDeviceToDevice, s));
    DBG_CK(cudaMemcpyAsync(dst->off.p, src->off.p, sizeof(int64_t) * (src->nnzb + 1), cudaMemcpyDeviceToDevice, s));
    if (src->nnzb) {
        DBG_CK(cudaMemcpyAsync(dst->col.p, src->col.p, sizeof(int32_t) * src->nnzb, cudaMemcpyDeviceToDevice, s));
        DBG_CK(cudaMemcpyAsync(dst->row.p, src->row.p, sizeof(int32_t) * src->nnzb, cudaMemcpyDeviceToDevice, s));
    }
    if (src->nel) DBG_CK(cudaMemcpyAsync(dst->data.p, src->data.p, sizeof(double) * src->nel, cudaMemcpyDeviceToDevice, s));
    dst->nnzb = src->nnzb;
    dst->nel = src->nel;
    dst->norms_valid = false;
    if (src->norms_valid && src->nnzb) {
        dst->norms.alloc(src->nnzb, s);
        DBG_CK(cudaMemcpyAsync(dst->norms.p, src->norms.p, sizeof(double) * src->nnzb, cudaMemcpyDeviceToDevice, s));
        dst->norms_valid = true;
    }
    dst->finalized = true;
}

void scale_shift(dbcsr_matrix_* m, double scale, double shift) {
    check_finalized(m);
    if (shift != 0.0) {
        DBuf<int64_t> missing;
        missing.alloc(1, m->stream);
        missing.zero();
        k_missing_diag<<<grid_for(m->nblk, 256), 256, 0, m->stream>>>(m->nblk, m->rp.p, m->col.p, missing.p);
        DBG_LAUNCH_CK();
        if (read_i64(missing.p, m->stream) != 0) fail(DBCSR_EINVAL, "scale_shift: a diagonal block is missing");
    }
    if (m->nnzb) {
        k_scale_shift<<<grid_for(m->nnzb, 8), 256, 0, m->stream>>>(m->nnzb, m->row.p, m->col.p, m->bs.p, m->off.p,
                                                                   m->data.p, scale, shift);
        DBG_LAUNCH_CK();
    }
    m->norms_valid = false;
}

void compact(dbcsr_matrix_* m, const int32_t* keep, const double* norms_in) {
    check_unplanned(m, "filter");
    cudaStream_t s = m->stream;
    const int64_t nb = m->nnzb;
    DBuf<int64_t> newidx;
    newidx.alloc(nb + 1, s);
    scan_exclusive(keep, newidx.p, nb, s);
    const int64_t nk = read_i64(newidx.p + nb, s);
    DBuf<int32_t> nrow, ncol;
    DBuf<int64_t> narea, noff, nrp;
    DBuf<double> nnorms;
    nrow.alloc(std::max<int64_t>(nk, 1), s);
    ncol.alloc(std::max<int64_t>(nk, 1), s);
    narea.alloc(std::max<int64_t>(nk, 1), s);
    noff.alloc(nk + 1, s);
    nrp.alloc(m->nblk + 1, s);
    if (norms_in) nnorms.alloc(std::max<int64_t>(nk, 1), s);
    if (nb) {
        k_compact_meta<<<grid_for(nb, 256), 256, 0, s>>>(nb, keep, newidx.p, m->row.p, m->col.p, m->bs.p, norms_in,
                                                         nrow.p, ncol.p, narea.p, norms_in ? nnorms.p : nullptr);
        DBG_LAUNCH_CK();
    }
    k_compact_rp<<<grid_for(m->nblk + 1, 256), 256, 0, s>>>(m->nblk, m->rp.p, newidx.p, nrp.p);
    DBG_LAUNCH_CK();
    scan_exclusive(narea.p, noff.p, nk, s);
    const int64_t nel = read_i64(noff.p + nk, s);
    DBuf<double> ndata;
    ndata.alloc(std::max<int64_t>(nel, 1), s);
    if (nb) {
        k_compact_data<<<grid_for(nb, 8), 256, 0, s>>>(nb, keep, newidx.p, m->off.p, noff.p, m->data.p, ndata.p);
        DBG_LAUNCH_CK();
    }
    m->rp = std::move(nrp);
    m->row = std::move(nrow);
    m->col = std::move(ncol);
    m->off = std::move(noff);
    m->data = std::move(ndata);
    m->nnzb = nk;
    m->nel = nel;
    if (norms_in) {
        m->norms = std::move(nnorms);
        m->norms_valid = true;
    } else {
        m->norms_valid = false;
    }
}

void filter_matrix(dbcsr_matrix_* m, double eps, const double* norms_in) {
    check_finalized(m);
    cudaStream_t s = m->stream;
    if (m->nnzb == 0) return;
    if (!norms_in) {
        ensure_norms(m);
        norms_in = m->norms.p;
    }
    DBuf<int32_t> keep;
    keep.alloc(m->nnzb, s);
    k_keep_norm<<<grid_for(m->nnzb, 256), 256, 0, s>>>(m->nnzb, m->row.p, m->col.p, norms_in, eps, keep.p);
    DBG_LAUNCH_CK();
    // norms_in may be owned by m: compact() replaces m->norms only after reading it
    compact(m, keep.p, norms_in);
}

}  // namespace dbg

// ------------------------------------------------------------------ C ABI
using dbg::fail;

namespace {
thread_local std::string g_last_error;

template <class F>
dbcsr_status guarded(F&& f) {
    try {
        f();
        g_last_error.clear();
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        g_last_error = e.what();
        return e.code;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return DBCSR_ENOMEM;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return DBCSR_EINVAL;
    }
}
}  // namespace

namespace {
// The matrix file: 8-byte magic "DBCSRGB1", int32 nblk, int32 0, int64 nnzb, int64 nel,
// then int32 blk_size[nblk], int64 row_ptr[nblk + 1], int32 col[nnzb], double data[nel],
// each in the host's byte order (little-endian on the supported hosts), and last the
// uint32 CRC-32 of all the bytes before it.
constexpr char kFileMagic[8] = {'D', 'B', 'C', 'S', 'R', 'G', 'B', '1'};

// CRC-32 as in IEEE 802.3 / zlib: reflected polynomial 0xEDB88320, register preset to all
// ones and inverted at the end; crc = crc32_update(crc, bytes) continues a running value.
uint32_t crc32_update(uint32_t crc, const void* buf, size_t len) {
    static const auto table = [] {
        std::array<uint32_t, 256> t{};
        for (uint32_t i = 0; i < 256; ++i) {
            uint32_t c = i;
            for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
            t[i] = c;
        }
        return t;
    }();
    const auto* p = static_cast<const unsigned char*>(buf);
    crc = ~crc;
    for (size_t i = 0; i < len; ++i) crc = table[(crc ^ p[i]) & 0xFFu] ^ (crc >> 8);
    return ~crc;
}

struct MatrixFile {
    int32_t nblk = 0;
    int64_t nnzb = 0, nel = 0;
    std::vector<int32_t> bs, col;
    std::vector<int64_t> rp;
    std::vector<double> data;
};

// Reads and checks a whole matrix file on the host (no device work).
MatrixFile read_matrix_file(const char* path) {
    using dbg::fail;
    if (!path) fail(DBCSR_EINVAL, "load: null path");
    std::FILE* f = std::fopen(path, "rb");
    if (!f) fail(DBCSR_EINVAL, std::string("load: cannot open ") + path);
    struct Closer {
        std::FILE* f;
        ~Closer() { std::fclose(f); }
    } closer{f};
    uint32_t crc = 0;
    auto read = [&](void* dst, size_t size, size_t count) {
        if (count && std::fread(dst, size, count, f) != count) fail(DBCSR_EINVAL, "load: file too short");
        crc = crc32_update(crc, dst, size * count);
    };
    if (std::fseek(f, 0, SEEK_END) != 0) fail(DBCSR_EINVAL, "load: cannot size the file");
    const int64_t fsize = (int64_t)std::ftell(f);
    if (fsize < 0 || std::fseek(f, 0, SEEK_SET) != 0) fail(DBCSR_EINVAL, "load: cannot size the file");
    char magic[8];
    int32_t nblk = 0, zero = 0;
    int64_t nnzb = 0, nel = 0;
    read(magic, 1, 8);
    if (std::memcmp(magic, kFileMagic, 8) != 0) fail(DBCSR_EINVAL, "load: not a matrix file");
    read(&nblk, sizeof nblk, 1);
    read(&zero, sizeof zero, 1);
    read(&nnzb, sizeof nnzb, 1);
    read(&nel, sizeof nel, 1);
    // sizes bounded by the file before any product is formed, then the exact length
    if (nblk < 1 || zero != 0 || nnzb < 0 || nel < 0 || nblk > fsize / 12 || nnzb > fsize / 4 || nel > fsize / 8)
        fail(DBCSR_EINVAL, "load: bad header");
    const int64_t expect = 32 + 4 * (int64_t)nblk + 8 * ((int64_t)nblk + 1) + 4 * nnzb + 8 * nel + 4;
    if (expect != fsize) fail(DBCSR_EINVAL, "load: file length does not match the header");
    MatrixFile m;
    m.nblk = nblk;
    m.nnzb = nnzb;
    m.nel = nel;
    m.bs.resize(nblk);
    m.rp.resize(nblk + 1);
    m.col.resize(nnzb);
    m.data.resize(nel);
    read(m.bs.data(), sizeof(int32_t), nblk);
    read(m.rp.data(), sizeof(int64_t), nblk + 1);
    read(m.col.data(), sizeof(int32_t), nnzb);
    read(m.data.data(), sizeof(double), nel);
    const uint32_t computed = crc;
    uint32_t stored = 0;
    read(&stored, sizeof stored, 1);
    if (stored != computed) fail(DBCSR_EINVAL, "load: checksum mismatch");
    for (int32_t b : m.bs)
        if (b < 1 || b > dbg::kMaxBlock) fail(DBCSR_EINVAL, "load: block edge outside [1, 32]");
    // the whole row-pointer array is checked before any column is read: a pointer past
    // nnzb in the middle of the array would otherwise index beyond the column vector
    if (m.rp[0] != 0 || m.rp[nblk] != nnzb) fail(DBCSR_EINVAL, "load: bad row pointers");
    for (int32_t i = 0; i < nblk; ++i)
        if (m.rp[i + 1] < m.rp[i] || m.rp[i + 1] > nnzb) fail(DBCSR_EINVAL, "load: bad row pointers");
    int64_t area = 0;
    for (int32_t i = 0; i < nblk; ++i) {
        for (int64_t q = m.rp[i]; q < m.rp[i + 1]; ++q) {
            const int32_t c = m.col[q];
            if (c < 0 || c >= nblk || (q > m.rp[i] && c <= m.col[q - 1]))
                fail(DBCSR_EINVAL, "load: columns out of range or not ascending");
            area += (int64_t)m.bs[i] * m.bs[c];
        }
    }
    if (area != nel) fail(DBCSR_EINVAL, "load: data size does not match the blocks");
    return m;
}
}  // namespace

namespace dbg {
[[noreturn]] void fail(dbcsr_status code, const std::string& msg) { throw Error(code, msg); }
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace dbg

extern "C" {

const char* dbcsr_last_error(void) { return g_last_error.c_str(); }

const char* dbcsr_version(void) { return "dbcsr_gb 0.1 (sm_103a)"; }

dbcsr_status dbcsr_pool_trim(uint64_t keep_bytes) {
    return guarded([&] { dbg::trim_pool(keep_bytes); });
}

dbcsr_status dbcsr_create(dbcsr_matrix* out, int32_t nblk, const int32_t* blk_size, void* stream) {
    return guarded([&] {
        if (!out || !blk_size || nblk < 1) fail(DBCSR_EINVAL, "create: need out, nblk >= 1 and blk_size");
        for (int32_t i = 0; i < nblk; ++i)
            if (blk_size[i] < 1 || blk_size[i] > dbg::kMaxBlock)
                fail(DBCSR_EINVAL, "create: block edge outside [1, 32] at " + std::to_string(i));
        auto* m = new dbcsr_matrix_();
        try {
            m->nblk = nblk;
            m->stream = (cudaStream_t)stream;
            m->h_bs.assign(blk_size, blk_size + nblk);
            m->n = std::accumulate(m->h_bs.begin(), m->h_bs.end(), (int64_t)0);
            m->bs.alloc(nblk, m->stream);
            DBG_CK(cudaMemcpyAsync(m->bs.p, blk_size, sizeof(int32_t) * nblk, cudaMemcpyHostToDevice, m->stream));
            DBG_CK(cudaStreamSynchronize(m->stream));
        } catch (...) {
            delete m;
            throw;
        }
        *out = m;
    });
}

int32_t dbcsr_matrix_groups(dbcsr_matrix m, int32_t* g_of, double* norms, int32_t* ngrp) {
    return guarded([&] {
        dbg::check_finalized(m);
        std::shared_ptr<dbg::Groups> g = dbg::build_groups(m);
        if (g_of && m->nblk)
            DBG_CK(cudaMemcpyAsync(g_of, g->g_of.p, sizeof(int32_t) * m->nblk, cudaMemcpyDeviceToHost, m->stream));
        if (norms && m->nnzb)
            DBG_CK(cudaMemcpyAsync(norms, m->norms.p, sizeof(double) * m->nnzb, cudaMemcpyDeviceToHost, m->stream));
        DBG_CK(cudaStreamSynchronize(m->stream));
        if (ngrp) *ngrp = g->ngrp;
    });
}

dbcsr_status dbcsr_destroy(dbcsr_matrix m) {
    return guarded([&] {
        if (!m) return;
        dbg::check_unplanned(m, "destroy");
        delete m;
    });
}

dbcsr_status dbcsr_put_values(dbcsr_matrix m, const double* data, int on_device) {
    return guarded([&] {
        dbg::check_finalized(m);
        if (!data && m->nel) dbg::fail(DBCSR_EINVAL, "put_values: null data");
        if (m->nel)
            DBG_CK(cudaMemcpyAsync(m->data.p, data, sizeof(double) * m->nel,
                                   on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m->stream));
        if (!on_device) DBG_CK(cudaStreamSynchronize(m->stream));
        m->norms_valid = false;
    });
}

// Every staged block is copied at once into a device staging pool (host sources
// through one cudaMemcpyAsync, so pinned host buffers move by DMA); the host-side records of
// the blocks are written while that copy runs.
static void stage(dbcsr_matrix m, int64_t n, const int32_t* rows, const int32_t* cols, const double* packed,
                  int on_device) {
    if (!m) fail(DBCSR_EINVAL, "null matrix handle");
    dbg::check_unplanned(m, "put_block");
    if (m->finalized) fail(DBCSR_ESTATE, "put_block: matrix already finalized");
    if (n < 0 || (n > 0 && (!rows || !cols || !packed))) fail(DBCSR_EINVAL, "put_blocks: null argument");
    const int32_t nblk = m->nblk;
    const int32_t* bs = m->h_bs.data();
    // per chunk: elements of its blocks (0 if an index is out of range) and a validity flag
    std::array<int64_t, 16> part{};
    std::array<int, 16> bad{};
    const int nt = dbg::host_chunks(n, [&](int c, int64_t b, int64_t e) {
        int64_t t = 0;
        bool x = false;
        for (int64_t i = b; i < e; ++i) {
            const int32_t r = rows[i], cl = cols[i];
            x |= (uint32_t)r >= (uint32_t)nblk || (uint32_t)cl >= (uint32_t)nblk;
            if (!x) t += (int64_t)bs[r] * bs[cl];
        }
        part[c] = t;
        bad[c] = x;
    });
    int64_t total = 0;
    for (int c = 0; c < nt; ++c) {
        if (bad[c]) fail(DBCSR_EINVAL, "put_block: block index out of range");
        total += part[c];
    }
    if (m->st_dev_used + total > m->st_dev.n) {
        const int64_t cap = std::max<int64_t>(m->st_dev.n + m->st_dev.n / 2, m->st_dev_used + total);
        dbg::DBuf<double> nb;
        nb.alloc(cap, m->stream);
        if (m->st_dev_used)
            DBG_CK(cudaMemcpyAsync(nb.p, m->st_dev.p, sizeof(double) * m->st_dev_used, cudaMemcpyDeviceToDevice,
                                   m->stream));
        m->st_dev = std::move(nb);
    }
    if (total)
        DBG_CK(cudaMemcpyAsync(m->st_dev.p + m->st_dev_used, packed, sizeof(double) * total,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m->stream));
    const size_t base = m->st_row.size();
    m->st_row.resize(base + n);
    m->st_col.resize(base + n);
    m->st_src.resize(base + n);
    std::array<int64_t, 16> start{};
    {
        int64_t acc = m->st_dev_used;
        for (int c = 0; c < nt; ++c) {
            start[c] = acc;
            acc += part[c];
        }
    }
    dbg::host_chunks(n, [&](int c, int64_t b, int64_t e) {
        int64_t at = start[c];
        for (int64_t i = b; i < e; ++i) {
            m->st_row[base + i] = rows[i];
            m->st_col[base + i] = cols[i];
            m->st_src[base + i] = at;
            at += (int64_t)bs[rows[i]] * bs[cols[i]];
        }
    });
    m->st_dev_used += total;
    DBG_CK(cudaStreamSynchronize(m->stream));   // the caller may reuse its buffers on return
}

dbcsr_status dbcsr_put_block(dbcsr_matrix m, int32_t row, int32_t col, const double* data, int on_device) {
    return guarded([&] { stage(m, 1, &row, &col, data, on_device); });
}

dbcsr_status dbcsr_put_blocks(dbcsr_matrix m, int64_t n, const int32_t* rows, const int32_t* cols,
                              const double* packed, int on_device) {
    return guarded([&] { stage(m, n, rows, cols, packed, on_device); });
}

dbcsr_status dbcsr_finalize(dbcsr_matrix m) {
    return guarded([&] {
        if (!m) fail(DBCSR_EINVAL, "null matrix handle");
        if (m->finalized) fail(DBCSR_ESTATE, "finalize: already finalized");
        const int64_t nb = (int64_t)m->st_row.size();
        const std::vector<int32_t>& sr = m->st_row;
        const std::vector<int32_t>& sc = m->st_col;
        // staged in strictly increasing (row, column) order: then no block repeats
        std::array<int, 16> unsorted{};
        dbg::host_chunks(nb, [&](int c, int64_t b, int64_t e) {
            bool u = false;
            for (int64_t i = std::max<int64_t>(b, 1); i < e && !u; ++i)
                u = !(sr[i - 1] < sr[i] || (sr[i - 1] == sr[i] && sc[i - 1] < sc[i]));
            unsorted[c] = u;
        });
        bool sorted = true;
        for (int c = 0; c < 16; ++c) sorted = sorted && !unsorted[c];
        std::vector<int64_t> order;
        if (!sorted) {
            order.resize(nb);
            std::iota(order.begin(), order.end(), 0);
            std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
                return sr[a] != sr[b] ? sr[a] < sr[b] : sc[a] < sc[b];
            });
            for (int64_t i = 1; i < nb; ++i) {
                const int64_t a = order[i - 1], b = order[i];
                if (sr[a] == sr[b] && sc[a] == sc[b])
                    fail(DBCSR_EINVAL, "finalize: duplicate block (" + std::to_string(sr[a]) + ", " +
                                           std::to_string(sc[a]) + ")");
            }
        }
        std::vector<int64_t> rp(m->nblk + 1, 0), off(nb + 1, 0), src(nb);
        std::vector<int32_t> col(nb), row(nb);
        // blocks in order, then their element offsets: per-chunk sums, then a fill from each
        // chunk's start
        std::array<int64_t, 16> part{};
        const int nt = dbg::host_chunks(nb, [&](int c, int64_t b, int64_t e) {
            int64_t t = 0;
            for (int64_t i = b; i < e; ++i) {
                const int64_t o = sorted ? i : order[i];
                row[i] = sr[o];
                col[i] = sc[o];
                src[i] = m->st_src[o];
                t += (int64_t)m->h_bs[row[i]] * m->h_bs[col[i]];
            }
            part[c] = t;
        });
        std::array<int64_t, 16> start{};
        for (int c = 1; c < nt; ++c) start[c] = start[c - 1] + part[c - 1];
        dbg::host_chunks(nb, [&](int c, int64_t b, int64_t e) {
            int64_t at = start[c];
            for (int64_t i = b; i < e; ++i) {
                off[i] = at;
                at += (int64_t)m->h_bs[row[i]] * m->h_bs[col[i]];
            }
        });
        off[nb] = nb ? start[nt - 1] + part[nt - 1] : 0;
        for (int64_t i = 0; i < nb; ++i) rp[row[i] + 1]++;
        for (int32_t I = 0; I < m->nblk; ++I) rp[I + 1] += rp[I];
        cudaStream_t s = m->stream;
        m->nnzb = nb;
        m->nel = off[nb];
        m->rp.alloc(m->nblk + 1, s);
        m->col.alloc(std::max<int64_t>(nb, 1), s);
        m->row.alloc(std::max<int64_t>(nb, 1), s);
        m->off.alloc(nb + 1, s);
        DBG_CK(cudaMemcpyAsync(m->rp.p, rp.data(), sizeof(int64_t) * (m->nblk + 1), cudaMemcpyHostToDevice, s));
        DBG_CK(cudaMemcpyAsync(m->off.p, off.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, s));
        if (nb) {
            DBG_CK(cudaMemcpyAsync(m->col.p, col.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s));
            DBG_CK(cudaMemcpyAsync(m->row.p, row.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s));
            std::array<int, 16> moved{};
            if (sorted)
                dbg::host_chunks(nb, [&](int c, int64_t b, int64_t e) {
                    bool x = false;
                    for (int64_t i = b; i < e && !x; ++i) x = src[i] != off[i];
                    moved[c] = x;
                });
            bool direct = sorted;
            for (int c = 0; c < 16; ++c) direct = direct && !moved[c];
            if (direct && m->st_dev_used == m->nel) {
                // staged in block-CSR order: the staging pool is the data
                m->data = std::move(m->st_dev);
            } else {
                m->data.alloc(std::max<int64_t>(m->nel, 1), s);
                dbg::DBuf<int64_t> dsrc;
                dsrc.alloc(nb, s);
                DBG_CK(cudaMemcpyAsync(dsrc.p, src.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, s));
                dbg::k_gather_blocks<<<dbg::grid_for(nb, 8), 256, 0, s>>>(nb, dsrc.p, m->st_dev.p, m->row.p, m->col.p,
                                                                           m->bs.p, m->off.p, m->data.p);
                DBG_LAUNCH_CK();
                DBG_CK(cudaStreamSynchronize(s));
            }
        }
        if (!m->data.p) m->data.alloc(1, s);    // no block: a one-element buffer, as for every matrix
        DBG_CK(cudaStreamSynchronize(s));
        m->st_row.clear(); m->st_row.shrink_to_fit();
        m->st_col.clear(); m->st_col.shrink_to_fit();
        m->st_src.clear(); m->st_src.shrink_to_fit();
        m->st_dev.release();
        m->st_dev_used = 0;
        m->norms_valid = false;
        m->finalized = true;
    });
}

dbcsr_status dbcsr_get_info(dbcsr_matrix m, int32_t* nblk, int64_t* nnzb, int64_t* nelem) {
    return guarded([&] {
        dbg::check_finalized(m);
        if (nblk) *nblk = m->nblk;
        if (nnzb) *nnzb = m->nnzb;
        if (nelem) *nelem = m->nel;
    });
}

dbcsr_status dbcsr_get_block(dbcsr_matrix m, int32_t row, int32_t col, double* out_host, int* present) {
    return guarded([&] {
        dbg::check_finalized(m);
        if (!present || row < 0 || col < 0 || row >= m->nblk || col >= m->nblk) fail(DBCSR_EINVAL, "get_block: bad argument");
        int64_t lohi[2];
        DBG_CK(cudaMemcpyAsync(lohi, m->rp.p + row, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, m->stream));
        DBG_CK(cudaStreamSynchronize(m->stream));
        std::vector<int32_t> cols(lohi[1] - lohi[0]);
        if (!cols.empty()) {
            DBG_CK(cudaMemcpyAsync(cols.data(), m->col.p + lohi[0], sizeof(int32_t) * cols.size(), cudaMemcpyDeviceToHost,
                                   m->stream));
            DBG_CK(cudaStreamSynchronize(m->stream));
        }
        auto it = std::lower_bound(cols.begin(), cols.end(), col);
        if (it == cols.end() || *it != col) {
            *present = 0;
            return;
        }
        const int64_t b = lohi[0] + (it - cols.begin());
        int64_t o;
        DBG_CK(cudaMemcpyAsync(&o, m->off.p + b, sizeof(int64_t), cudaMemcpyDeviceToHost, m->stream));
        DBG_CK(cudaStreamSynchronize(m->stream));
        if (out_host) {
            DBG_CK(cudaMemcpyAsync(out_host, m->data.p + o, sizeof(double) * m->h_bs[row] * m->h_bs[col],
                                   cudaMemcpyDeviceToHost, m->stream));
            DBG_CK(cudaStreamSynchronize(m->stream));
        }
        *present = 1;
    });
}

dbcsr_status dbcsr_export(dbcsr_matrix m, int64_t* row_ptr, int32_t* col, double* data) {
    return guarded([&] {
        dbg::check_finalized(m);
        cudaStream_t s = m->stream;
        if (row_ptr) DBG_CK(cudaMemcpyAsync(row_ptr, m->rp.p, sizeof(int64_t) * (m->nblk + 1), cudaMemcpyDeviceToHost, s));
        if (col && m->nnzb) DBG_CK(cudaMemcpyAsync(col, m->col.p, sizeof(int32_t) * m->nnzb, cudaMemcpyDeviceToHost, s));
        if (data && m->nel) DBG_CK(cudaMemcpyAsync(data, m->data.p, sizeof(double) * m->nel, cudaMemcpyDeviceToHost, s));
        DBG_CK(cudaStreamSynchronize(s));
    });
}

dbcsr_status dbcsr_copy(dbcsr_matrix dst, dbcsr_matrix src) {
    return guarded([&] {
        if (!dst) fail(DBCSR_EINVAL, "null matrix handle");
        dbg::copy_matrix(dst, src);
    });
}

dbcsr_status dbcsr_scale_shift(dbcsr_matrix m, double scale, double shift) {
    return guarded([&] { dbg::scale_shift(m, scale, shift); });
}

dbcsr_status dbcsr_add(double alpha, dbcsr_matrix A, double beta, dbcsr_matrix B) {
    return guarded([&] { dbg::add(A, alpha, B, beta); });
}

dbcsr_status dbcsr_filter(dbcsr_matrix m, double eps) {
    return guarded([&] { dbg::filter_matrix(m, eps, nullptr); });
}

dbcsr_status dbcsr_multiply(double alpha, dbcsr_matrix A, dbcsr_matrix B, double beta, dbcsr_matrix C,
                            double eps_filter, int32_t prec, dbcsr_mult_stats* stats) {
    return guarded([&] { dbg::multiply(alpha, A, B, beta, C, eps_filter, prec, stats, stats != nullptr); });
}

dbcsr_status dbcsr_trace(dbcsr_matrix A, double* out) {
    return guarded([&] {
        if (!out) fail(DBCSR_EINVAL, "trace: null output");
        *out = dbg::trace(A);
    });
}

dbcsr_status dbcsr_trace_product(dbcsr_matrix A, dbcsr_matrix B, double* out) {
    return guarded([&] {
        if (!out) fail(DBCSR_EINVAL, "trace_product: null output");
        *out = dbg::trace_product(A, B);
    });
}

dbcsr_status dbcsr_gershgorin(dbcsr_matrix A, double mu, double* out) {
    return guarded([&] {
        if (!out) fail(DBCSR_EINVAL, "gershgorin: null output");
        *out = dbg::gershgorin(A, mu);
    });
}

dbcsr_status dbcsr_sign_iterate(dbcsr_matrix H, double mu, const dbcsr_sign_opts* opts, dbcsr_matrix P_out,
                                dbcsr_sign_report* rep) {
    dbcsr_status st = DBCSR_OK;
    dbcsr_status g = guarded([&] { st = dbg::sign_iterate(H, mu, opts, P_out, rep); });
    if (g != DBCSR_OK) return g;
    if (st != DBCSR_OK) g_last_error = "sign iteration did not reach the tolerance";
    return st;
}

dbcsr_status dbcsr_sign_iterate_resume(dbcsr_matrix H, dbcsr_matrix X, const dbcsr_sign_report* prev,
                                       const dbcsr_sign_opts* opts, dbcsr_matrix P_out, dbcsr_sign_report* rep) {
    dbcsr_status st = DBCSR_OK;
    dbcsr_status g = guarded([&] { st = dbg::sign_iterate_resume(H, X, prev, opts, P_out, rep); });
    if (g != DBCSR_OK) return g;
    if (st != DBCSR_OK) g_last_error = "sign iteration did not reach the tolerance";
    return st;
}

dbcsr_status dbcsr_inverse_sqrt(dbcsr_matrix S, const dbcsr_sign_opts* opts, dbcsr_matrix S_invsqrt,
                                dbcsr_matrix S_sqrt, dbcsr_sign_report* rep) {
    dbcsr_status st = DBCSR_OK;
    dbcsr_status g = guarded([&] { st = dbg::inverse_sqrt(S, opts, S_invsqrt, S_sqrt, rep); });
    if (g != DBCSR_OK) return g;
    if (st != DBCSR_OK) g_last_error = "square-root iteration did not reach the tolerance";
    return st;
}

dbcsr_status dbcsr_inverse_hotelling(dbcsr_matrix A, const dbcsr_sign_opts* opts, dbcsr_matrix A_inv,
                                     dbcsr_sign_report* rep) {
    dbcsr_status st = DBCSR_OK;
    dbcsr_status g = guarded([&] { st = dbg::inverse_hotelling(A, opts, A_inv, rep); });
    if (g != DBCSR_OK) return g;
    if (st != DBCSR_OK) g_last_error = "Hotelling iteration did not reach the tolerance";
    return st;
}

dbcsr_status dbcsr_sign_iterate_nonorth(dbcsr_matrix K, dbcsr_matrix S, double mu, const dbcsr_sign_opts* opts,
                                        dbcsr_matrix P_out, dbcsr_sign_report* rep, dbcsr_sign_report* rep_sqrt) {
    dbcsr_status st = DBCSR_OK;
    dbcsr_status g = guarded([&] { st = dbg::sign_iterate_nonorth(K, S, mu, opts, P_out, rep, rep_sqrt); });
    if (g != DBCSR_OK) return g;
    if (st != DBCSR_OK) g_last_error = "an iteration did not reach the tolerance";
    return st;
}

dbcsr_status dbcsr_purify(dbcsr_matrix H, double n_occ, int32_t method, const dbcsr_sign_opts* opts,
                          dbcsr_matrix P_out, dbcsr_sign_report* rep) {
    dbcsr_status st = DBCSR_OK;
    dbcsr_status g = guarded([&] { st = dbg::purify(H, n_occ, method, opts, P_out, rep); });
    if (g != DBCSR_OK) return g;
    if (st != DBCSR_OK) g_last_error = "purification did not reach the tolerance";
    return st;
}

dbcsr_status dbcsr_sign_mu_search(dbcsr_matrix H, double n_occ, double mu_lo, double mu_hi, const dbcsr_sign_opts* opts,
                                  dbcsr_matrix P_out, double* mu_out, int32_t* evaluations, dbcsr_sign_report* rep) {
    dbcsr_status st = DBCSR_OK;
    dbcsr_status g = guarded([&] { st = dbg::sign_mu_search(H, n_occ, mu_lo, mu_hi, opts, P_out, mu_out, evaluations, rep); });
    if (g != DBCSR_OK) return g;
    if (st != DBCSR_OK) g_last_error = "no chemical potential with the requested occupation was reached";
    return st;
}

dbcsr_status dbcsr_submatrix_sign(dbcsr_matrix H, double mu, const dbcsr_sign_opts* opts, dbcsr_matrix P_out,
                                  dbcsr_sign_report* rep) {
    dbcsr_status st = DBCSR_OK;
    dbcsr_status g = guarded([&] { st = dbg::submatrix_sign(H, mu, opts, P_out, rep); });
    if (g != DBCSR_OK) return g;
    if (st != DBCSR_OK) g_last_error = "a submatrix did not reach the tolerance";
    return st;
}

dbcsr_status dbcsr_save(dbcsr_matrix m, const char* path) {
    return guarded([&] {
        dbg::check_finalized(m);
        if (!path) fail(DBCSR_EINVAL, "save: null path");
        std::vector<int64_t> rp(m->nblk + 1);
        std::vector<int32_t> col(std::max<int64_t>(m->nnzb, 1));
        std::vector<double> data(std::max<int64_t>(m->nel, 1));
        cudaStream_t s = m->stream;
        DBG_CK(cudaMemcpyAsync(rp.data(), m->rp.p, sizeof(int64_t) * (m->nblk + 1), cudaMemcpyDeviceToHost, s));
        if (m->nnzb) DBG_CK(cudaMemcpyAsync(col.data(), m->col.p, sizeof(int32_t) * m->nnzb, cudaMemcpyDeviceToHost, s));
        if (m->nel) DBG_CK(cudaMemcpyAsync(data.data(), m->data.p, sizeof(double) * m->nel, cudaMemcpyDeviceToHost, s));
        DBG_CK(cudaStreamSynchronize(s));
        std::FILE* f = std::fopen(path, "wb");
        if (!f) fail(DBCSR_EINVAL, std::string("save: cannot open ") + path);
        const int32_t zero = 0;
        uint32_t crc = 0;
        auto put = [&](const void* src, size_t size, size_t count) {
            crc = crc32_update(crc, src, size * count);
            return count == 0 || std::fwrite(src, size, count, f) == count;
        };
        bool ok = put(kFileMagic, 1, 8) && put(&m->nblk, sizeof(int32_t), 1) && put(&zero, sizeof(int32_t), 1) &&
                  put(&m->nnzb, sizeof(int64_t), 1) && put(&m->nel, sizeof(int64_t), 1) &&
                  put(m->h_bs.data(), sizeof(int32_t), m->nblk) && put(rp.data(), sizeof(int64_t), m->nblk + 1) &&
                  put(col.data(), sizeof(int32_t), m->nnzb) && put(data.data(), sizeof(double), m->nel);
        const uint32_t final_crc = crc;
        ok = ok && std::fwrite(&final_crc, sizeof final_crc, 1, f) == 1;
        ok = (std::fclose(f) == 0) && ok;
        if (!ok) fail(DBCSR_EINVAL, std::string("save: write failed on ") + path);
    });
}

dbcsr_status dbcsr_file_info(const char* path, int32_t* nblk, int64_t* nnzb, int64_t* nel) {
    return guarded([&] {
        const MatrixFile mf = read_matrix_file(path);
        if (nblk) *nblk = mf.nblk;
        if (nnzb) *nnzb = mf.nnzb;
        if (nel) *nel = mf.nel;
    });
}

dbcsr_status dbcsr_load(dbcsr_matrix* out, const char* path, void* stream) {
    return guarded([&] {
        if (!out) fail(DBCSR_EINVAL, "load: null output handle");
        const MatrixFile mf = read_matrix_file(path);
        dbcsr_matrix m = nullptr;
        dbcsr_status st = dbcsr_create(&m, mf.nblk, mf.bs.data(), stream);
        if (st != DBCSR_OK) fail(st, g_last_error);
        try {
            std::vector<int32_t> rows(std::max<int64_t>(mf.nnzb, 1));
            for (int32_t i = 0; i < mf.nblk; ++i)
                for (int64_t q = mf.rp[i]; q < mf.rp[i + 1]; ++q) rows[q] = i;
            stage(m, mf.nnzb, rows.data(), mf.col.data(), mf.data.data(), 0);
            st = dbcsr_finalize(m);
            if (st != DBCSR_OK) fail(st, g_last_error);
        } catch (...) {
            dbcsr_destroy(m);
            throw;
        }
        *out = m;
    });
}

}  // extern "C"
