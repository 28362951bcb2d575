// Batched dense products of the submatrix method (section "Submatrix Method": each
// submatrix is purified densely), C[b] = alpha A[b] B[b] + beta C[b] for a batch of n x n
// row-major matrices, in the library's own kernels:
//
//   * FP32 storage on the 5th-generation tensor cores (tcgen05.mma kind::tf32, FP32
//     accumulators in tensor memory).  Plain TF32 rounds each operand to 10 stored bits;
//     split TF32 (x = hi + lo, both TF32, three products hi*hi + hi*lo + lo*hi) carries about
//     21 bits, close to FP32 arithmetic.  Operands are first packed into the K-major
//     no-swizzle layout of tc05.cuh (B transposed), 128-row tiles of A and up-to-256-row tiles
//     of B, K in steps of 8; one CTA per C tile streams K in stages of two steps with bulk
//     copies, one thread issues the MMAs (M = 128, N = the B tile's rows, K = 8), and four
//     warps write the accumulator back (one row each).
//   * FP64 storage on the FP64 pipe: 64 x 64 C tiles, 16-wide K slices in shared memory, a
//     4 x 4 register tile per thread.  GB300's FP64 rate is low enough (about 3.5 flops per
//     SM cycle) that the FMA loop, not memory, bounds it.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "tc05.cuh"

namespace dbg {
namespace {

constexpr int kDM = 128;                 // M of the MMA and rows of an A tile
constexpr int kDNMax = 256;              // rows of the widest B tile (N of the MMA)
constexpr int kDStepK = 8;               // TF32 elements per MMA K step (32 bytes)
constexpr int kDRunParts = 2;            // K steps x parts per stage: two steps plain, one step split
constexpr int kDStages = 4;
constexpr int kDStageBytes = kDRunParts * 2 * (kDM + kDNMax) * 16;   // 24 KB: two CTAs fit an SM
constexpr int kDEpiCols = 64;            // accumulator columns staged per pass of the epilogue
constexpr int kDThreads = 128;
constexpr long long kDWaitLimit = 4000000000ll;

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Packs a batch of n x n row-major matrices into tiles: tile (b, t) holds rows
// [t R, t R + R) of M[b] (transpose = 0) or of M[b]^T (transpose = 1), all K = kpad columns,
// as K steps of 8: per step np parts (hi, lo) x 2 chunks x R rows x 16 bytes.  Zero outside n.
// A thread writes one 16-byte chunk row (4 consecutive K elements of one row), threads in the
// order of the packed layout, so the writes are contiguous.
__global__ void k_dense_pack(int64_t total, int n, int kpad, int R, int ntiles, int np, int transpose,
                             const float* __restrict__ M, float* __restrict__ out) {
    const int nsteps = kpad / kDStepK;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        // e enumerates (b, t, step, chunk, row r) with r fastest
        const int r = (int)(e % R);
        int64_t rest = e / R;
        const int ch = (int)(rest % 2);
        rest /= 2;
        const int st = (int)(rest % nsteps);
        rest /= nsteps;
        const int t = (int)(rest % ntiles);
        const int64_t b = rest / ntiles;
        const int row = t * R + r, c0 = st * kDStepK + ch * 4;
        float x[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = c0 + q;
            x[q] = (row < n && c < n) ? (transpose ? M[b * n * n + (int64_t)c * n + row] : M[b * n * n + (int64_t)row * n + c])
                                      : 0.f;
        }
        const int64_t step_bytes = (int64_t)np * 2 * R * 16;
        uint8_t* base = reinterpret_cast<uint8_t*>(out) + ((b * ntiles + t) * nsteps + st) * step_bytes + ch * (R * 16) +
                        r * 16;
        float4 hi = make_float4(to_tf32(x[0]), to_tf32(x[1]), to_tf32(x[2]), to_tf32(x[3]));
        *reinterpret_cast<float4*>(base) = hi;
        if (np == 2)
            *reinterpret_cast<float4*>(base + 2 * R * 16) =
                make_float4(to_tf32(x[0] - hi.x), to_tf32(x[1] - hi.y), to_tf32(x[2] - hi.z), to_tf32(x[3] - hi.w));
    }
}

struct DenseArgs {
    int n, kpad, ntm, ntn, NT, np;       // NT: rows of every B tile (N of the MMA)
    const uint8_t* a_pack; const uint8_t* b_pack;
    float alpha, beta;
    float* C;
    int* err;
};

struct DenseShared {
    alignas(1024) uint8_t stage[kDStages][kDStageBytes];   // after the K loop: the epilogue's staging
    uint64_t full[kDStages], empty[kDStages], done;
    uint32_t tmem_base;
};

__global__ void __launch_bounds__(kDThreads, 2) k_dense_tf32(DenseArgs D) {
    extern __shared__ __align__(1024) uint8_t d_dyn[];
    DenseShared& S = *reinterpret_cast<DenseShared*>((reinterpret_cast<uintptr_t>(d_dyn) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tm = blockIdx.x, tn = blockIdx.y;
    const int64_t b = blockIdx.z;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kDStages; ++i) {
            tc::mbar_init(&S.full[i], 1);
            tc::mbar_init(&S.empty[i], 1);
        }
        tc::mbar_init(&S.done, 1);
        tc::fence_barrier_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&S.tmem_base, kDNMax);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = S.tmem_base;
    const int np = D.np, NT = D.NT;
    const int64_t sa_step = (int64_t)np * 2 * kDM * 16, sb_step = (int64_t)np * 2 * NT * 16;
    const int nk = D.kpad / kDStepK;
    const int run = kDRunParts / np;                      // K steps per stage
    const int nstage = (nk + run - 1) / run;
    const uint8_t* pa = D.a_pack + (b * D.ntm + tm) * (int64_t)nk * sa_step;
    const uint8_t* pb = D.b_pack + (b * D.ntn + tn) * (int64_t)nk * sb_step;
    bool ok = true;
    if (threadIdx.x == 0) {
        // one thread streams the K stages and issues the MMAs; a stage is refilled once the
        // MMAs that read it have completed
        int issued = 0;
        auto issue = [&](int s) {
            const int slot = s % kDStages;
            issued = s + 1;
            const int k0 = s * run, len = min(run, nk - k0);
            tc::mbar_arrive_expect_tx(&S.full[slot], (uint32_t)(len * (sa_step + sb_step)));
            tc::bulk_g2s(S.stage[slot], pa + k0 * sa_step, (uint32_t)(len * sa_step), &S.full[slot]);
            tc::bulk_g2s(S.stage[slot] + len * sa_step, pb + k0 * sb_step, (uint32_t)(len * sb_step), &S.full[slot]);
        };
        for (int s = 0; s < min(kDStages, nstage); ++s) issue(s);
        const uint32_t idesc = tc::instr_desc(2, kDM, NT);
        uint32_t accumulate = 0;
        for (int s = 0; s < nstage && ok; ++s) {
            const int slot = s % kDStages;
            const uint32_t phase = (uint32_t)(s / kDStages) & 1u;
            if (!tc::mbar_wait(&S.full[slot], phase, kDWaitLimit)) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const int len = min(run, nk - s * run);
            const uint32_t s0 = tc::smem_u32(S.stage[slot]);
            for (int j = 0; j < len; ++j) {
                const uint32_t sa = s0 + (uint32_t)(j * sa_step), sb = s0 + (uint32_t)(len * sa_step + j * sb_step);
                const uint64_t ah = tc::smem_desc(sa, kDM * 16, 128), bh = tc::smem_desc(sb, NT * 16, 128);
                tc::mma_tf32(tmem, ah, bh, idesc, accumulate);
                accumulate = 1;
                if (np == 2) {
                    const uint64_t al = tc::smem_desc(sa + 2 * kDM * 16, kDM * 16, 128);
                    const uint64_t bl = tc::smem_desc(sb + 2 * NT * 16, NT * 16, 128);
                    tc::mma_tf32(tmem, ah, bl, idesc, 1);
                    tc::mma_tf32(tmem, al, bh, idesc, 1);
                }
            }
            tc::mma_commit(&S.empty[slot]);
            // refill the previous stage's slot: its MMAs ran before these, which keep the tensor
            // cores busy while this thread waits
            const int pr = s - 1;
            if (pr >= 0 && pr + kDStages < nstage) {
                const int pslot = pr % kDStages;
                if (!tc::mbar_wait(&S.empty[pslot], (uint32_t)(pr / kDStages) & 1u, kDWaitLimit)) {
                    ok = false;
                    break;
                }
                issue(pr + kDStages);
            }
        }
        tc::mma_commit(&S.done);
        if (!tc::mbar_wait(&S.done, 0, kDWaitLimit)) ok = false;
        // copies still landing (after a wait that ran out) are waited for, bounded, before exit
        for (int s = max(0, issued - kDStages); s < issued; ++s) {
            const int slot = s % kDStages;
            tc::mbar_wait(&S.full[slot], (uint32_t)(s / kDStages) & 1u, kDWaitLimit);
        }
        if (!ok) atomicExch(D.err, 1);
    }
    __syncthreads();
    tc::fence_after_sync();
    // epilogue, kDEpiCols columns per pass: thread r reads row r of the accumulator (TMEM lane
    // r) into shared memory (the stage ring is idle now: every copy landed and every MMA
    // completed), then each warp writes whole row segments, lanes over consecutive columns
    float* T = reinterpret_cast<float*>(S.stage[0]);
    constexpr int kTS = kDEpiCols + 1;                    // odd stride: no bank conflicts
    float* Cb = D.C + b * D.n * D.n;
    const int r0 = tm * kDM;
    for (int c0 = 0; c0 < NT; c0 += kDEpiCols) {
        const int cw = min(kDEpiCols, NT - c0);
        for (int c = 0; c < cw; c += 16) {
            float v[16];
            tc::tmem_ld16(tmem + (uint32_t)(c0 + c) + ((uint32_t)(32 * warp) << 16), v);
#pragma unroll
            for (int x = 0; x < 16; ++x) T[threadIdx.x * kTS + c + x] = v[x];
        }
        __syncthreads();
        const int col0 = tn * NT + c0;
        const int ncol = min(cw, D.n - col0);
        for (int r = warp; r < kDM; r += kDThreads / 32) {
            const int row = r0 + r;
            if (row >= D.n) break;
            float* out = Cb + (int64_t)row * D.n + col0;
            for (int c = lane; c < ncol; c += 32) {
                const float v = D.alpha * T[r * kTS + c];
                out[c] = D.beta == 0.f ? v : v + D.beta * out[c];
            }
        }
        __syncthreads();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kDNMax);
    }
}

// FP64: C tile 64 x 64 per CTA of 256 threads, each a 4 x 4 register tile; K in slices of 16
// through shared memory.
constexpr int kF = 64, kFK = 16;

__global__ void __launch_bounds__(256) k_dense_f64(int n, double alpha, const double* __restrict__ A,
                                                   const double* __restrict__ B, double beta, double* __restrict__ C) {
    __shared__ double sa[kFK][kF + 1];   // A slice transposed: sa[k][i]
    __shared__ double sb[kFK][kF + 1];
    const int64_t b = blockIdx.z;
    const int i0 = blockIdx.y * kF, j0 = blockIdx.x * kF;
    const double* a = A + b * n * n;
    const double* bb = B + b * n * n;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < n; k0 += kFK) {
        for (int e = threadIdx.x; e < kF * kFK; e += 256) {
            const int r = e / kFK, c = e % kFK;          // A: row i0 + r, column k0 + c
            sa[c][r] = (i0 + r < n && k0 + c < n) ? a[(int64_t)(i0 + r) * n + k0 + c] : 0.0;
            const int kr = e / kF, jc = e % kF;          // B: row k0 + kr, column j0 + jc
            sb[kr][jc] = (k0 + kr < n && j0 + jc < n) ? bb[(int64_t)(k0 + kr) * n + j0 + jc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kFK; ++k) {
            double av[4], bv[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                av[x] = sa[k][ty + 16 * x];
                bv[x] = sb[k][tx + 16 * x];
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fma(av[x], bv[y], acc[x][y]);
        }
        __syncthreads();
    }
    double* c = C + b * n * n;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int i = i0 + ty + 16 * x, j = j0 + tx + 16 * y;
            if (i < n && j < n) {
                const int64_t p = (int64_t)i * n + j;
                c[p] = beta == 0.0 ? alpha * acc[x][y] : alpha * acc[x][y] + beta * c[p];
            }
        }
}

}  // namespace

void dense_gemm_f64(int64_t nb, int n, double alpha, const double* A, const double* B, double beta, double* C,
                    cudaStream_t s) {
    if (nb > 0 && n > 0 && nb > 65535) fail(DBCSR_ECAPACITY, "dense_gemm: more than 65535 matrices in one batch");
    if (nb <= 0 || n <= 0) return;
    if (nb > 65535) fail(DBCSR_ECAPACITY, "dense_gemm: more than 65535 matrices in one batch");
    const dim3 grid((unsigned)ceil_div(n, kF), (unsigned)ceil_div(n, kF), (unsigned)nb);
    k_dense_f64<<<grid, 256, 0, s>>>(n, alpha, A, B, beta, C);
    DBG_LAUNCH_CK();
}

void dense_gemm_tf32(int64_t nb, int n, float alpha, const float* A, const float* B, float beta, float* C, bool split,
                     cudaStream_t s) {
    if (nb <= 0 || n <= 0) return;
    if (nb > 65535) fail(DBCSR_ECAPACITY, "dense_gemm: more than 65535 matrices in one batch");
    const int np = split ? 2 : 1;
    const int kpad = (int)ceil_div(n, kDStepK) * kDStepK;
    const int ntm = (int)ceil_div(n, kDM);
    // N tiles of equal width (a multiple of 16, at most 256)
    const int ntn = (int)ceil_div(n, kDNMax);
    const int NT = (int)ceil_div(ceil_div(n, ntn), 16) * 16;
    const int64_t a_bytes = nb * ntm * (int64_t)(kpad / kDStepK) * np * 2 * kDM * 16;
    const int64_t b_bytes = nb * ntn * (int64_t)(kpad / kDStepK) * np * 2 * NT * 16;
    DBuf<float> pa, pb;
    DBuf<int> err;
    pa.alloc(a_bytes / 4, s);
    pb.alloc(b_bytes / 4, s);
    err.alloc(1, s);
    err.zero();
    const int64_t ta = nb * ntm * (int64_t)kDM * (kpad / 4), tb = nb * ntn * (int64_t)NT * (kpad / 4);
    k_dense_pack<<<grid_for(ta, 256), 256, 0, s>>>(ta, n, kpad, kDM, ntm, np, 0, A, pa.p);
    DBG_LAUNCH_CK();
    k_dense_pack<<<grid_for(tb, 256), 256, 0, s>>>(tb, n, kpad, NT, ntn, np, 1, B, pb.p);
    DBG_LAUNCH_CK();
    DenseArgs d{n, kpad, ntm, ntn, NT, np, reinterpret_cast<const uint8_t*>(pa.p),
                reinterpret_cast<const uint8_t*>(pb.p), alpha, beta, C, err.p};
    const size_t sm = sizeof(DenseShared) + 1024;
    allow_dyn_smem(k_dense_tf32, sm);
    k_dense_tf32<<<dim3((unsigned)ntm, (unsigned)ntn, (unsigned)nb), kDThreads, sm, s>>>(d);
    DBG_LAUNCH_CK();
    int e = 0;
    DBG_CK(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    DBG_CK(cudaStreamSynchronize(s));
    if (e) fail(DBCSR_ETIMEOUT, "dense_gemm: a wait of the tensor-core kernel ran out");
}

}  // namespace dbg

extern "C" dbcsr_status dbcsr_dense_multiply(int32_t prec, int64_t nb, int32_t n, double alpha, const void* A,
                                             const void* B, double beta, void* C, void* stream) {
    try {
        if (nb < 0 || n < 0 || (nb > 0 && n > 0 && (!A || !B || !C)))
            dbg::fail(DBCSR_EINVAL, "dense_multiply: bad argument");
        cudaStream_t s = (cudaStream_t)stream;
        if (prec == DBCSR_FP64) {
            dbg::dense_gemm_f64(nb, n, alpha, (const double*)A, (const double*)B, beta, (double*)C, s);
            DBG_CK(cudaStreamSynchronize(s));
        } else if (prec == DBCSR_TF32 || prec == DBCSR_TF32X3) {
            dbg::dense_gemm_tf32(nb, n, (float)alpha, (const float*)A, (const float*)B, (float)beta, (float*)C,
                                 prec == DBCSR_TF32X3, s);
        } else {
            dbg::fail(DBCSR_EINVAL, "dense_multiply: prec must be DBCSR_FP64, DBCSR_TF32 or DBCSR_TF32X3");
        }
        dbg::set_last_error("");
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    }
}
