// Batched dense products of the submatrix method (section "Submatrix Method": each
// submatrix is purified densely), C[b] = alpha A[b] B[b] + beta C[b] for a batch of n x n
// row-major matrices, in the library's own kernels:
//
//   * FP32 storage on the 5th-generation tensor cores (tcgen05.mma kind::tf32, FP32
//     accumulators in tensor memory).  Plain TF32 keeps 10 stored bits of each operand (the
//     tensor cores drop the low 13); split TF32 (hi = x so truncated, lo = x - hi likewise,
//     three products hi*hi + hi*lo + lo*hi) carries about 20 bits, close to FP32 arithmetic.  Operands are first packed into the K-major
//     no-swizzle layout of tc05.cuh (B transposed), 128-row tiles of A and up-to-256-row tiles
//     of B, K in steps of 8; one CTA per C tile streams K in stages of two steps with bulk
//     copies, one thread issues the MMAs (M = 128, N = the B tile's rows, K = 8), and four
//     warps write the accumulator back (one row each).
//   * FP64 storage on the FP64 pipe: 64 x 64 C tiles, 16-wide K slices in shared memory, a
//     4 x 4 register tile per thread.  GB300's FP64 rate is low enough (about 3.5 flops per
//     SM cycle) that the FMA loop, not memory, bounds it.
#include <algorithm>
#include <cstdint>

#include <cuda.h>
#include <cudaTypedefs.h>

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

// TF32 as the tensor cores read an FP32 operand: the 13 low mantissa bits dropped (truncation
// toward zero).  Both paths store operands this way, so a stored value is what is multiplied.
__device__ __forceinline__ float to_tf32(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

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

// ---------------------------------------------------------------- TF32 from tensor-map loads
// For n a multiple of 4 the operands need no pack pass: a 3-D tensor map (columns, rows,
// matrix) over A and one over B^T (B transposed once per product) bring 16 K columns of a
// 128-row A tile and of an N-row B tile per stage straight from the FP32 matrices, in the
// 64-byte swizzled K-major layout, and the MMAs read them as they are (as TF32).  For split
// operands four converter warps write lo = x - tf32(x) of every stage into a second buffer;
// one thread issues the MMAs (two K = 8 steps per stage); the four warps then write the
// accumulator back.
constexpr int kTK = 16;                                  // K columns per stage (64-byte rows)
constexpr int kTStages = 4;
constexpr int kTStageBytes = (kDM + kDNMax) * kTK * 4;  // 24 KB: A 8 KB, B up to 16 KB
constexpr int kTThreads = 192;                           // producer, MMA, 4 converter / epilogue warps

template <bool SPLIT>
struct TmaShared {
    alignas(1024) uint8_t x[kTStages][kTStageBytes];
    alignas(1024) uint8_t lo[SPLIT ? kTStages : 1][SPLIT ? kTStageBytes : 16];
    uint64_t full[kTStages], conv[kTStages], empty[kTStages], done;
    uint32_t tmem_base;
    int abort;
};

struct TmaArgs {
    int n, ntm, ntn, NT;
    float alpha, beta;
    float* C;
    int* err;
};

template <bool SPLIT>
__global__ void __launch_bounds__(kTThreads, 1)
    k_dense_tf32_tma(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_bt, TmaArgs D) {
    extern __shared__ __align__(1024) uint8_t t_dyn[];
    auto& S = *reinterpret_cast<TmaShared<SPLIT>*>((reinterpret_cast<uintptr_t>(t_dyn) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tm = blockIdx.x, tn = blockIdx.y, b = blockIdx.z;
    const int NT = D.NT;
    const int a_bytes = kDM * kTK * 4, b_bytes = NT * kTK * 4;
    const int nstage = (D.n + kTK - 1) / kTK;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kTStages; ++i) {
            tc::mbar_init(&S.full[i], 1);
            tc::mbar_init(&S.conv[i], 128);
            tc::mbar_init(&S.empty[i], 1);
        }
        tc::mbar_init(&S.done, 1);
        S.abort = 0;
        tc::fence_barrier_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(&S.tmem_base, kDNMax);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = S.tmem_base;
    if (warp == 0) {
        // ---- producer (lane 0): a stage is refilled once the MMAs that read it completed
        if (lane == 0) {
            int issued = 0;
            for (int s = 0; s < nstage; ++s) {
                const int slot = s % kTStages;
                if (s >= kTStages &&
                    !tc::mbar_wait(&S.empty[slot], (uint32_t)((s / kTStages) - 1) & 1u, kDWaitLimit)) {
                    *(volatile int*)&S.abort = 1;
                    atomicExch(D.err, 1);
                    break;
                }
                if (*(volatile int*)&S.abort) break;
                tc::mbar_arrive_expect_tx(&S.full[slot], (uint32_t)(a_bytes + b_bytes));
                tc::tma_load3d(S.x[slot], &map_a, s * kTK, tm * kDM, b, &S.full[slot]);
                tc::tma_load3d(S.x[slot] + a_bytes, &map_bt, s * kTK, tn * NT, b, &S.full[slot]);
                issued = s + 1;
            }
            // no copy may still be landing when the CTA exits
            for (int s = max(0, issued - kTStages); s < issued; ++s)
                tc::mbar_wait(&S.full[s % kTStages], (uint32_t)(s / kTStages) & 1u, kDWaitLimit);
        }
    } else if (warp == 1) {
        // ---- MMA issuer (lane 0)
        if (lane == 0) {
            const uint32_t idesc = tc::instr_desc(2, kDM, NT);
            bool ok = true;
            for (int s = 0; s < nstage && ok; ++s) {
                const int slot = s % kTStages;
                const uint32_t ph = (uint32_t)(s / kTStages) & 1u;
                if (!tc::mbar_wait(SPLIT ? &S.conv[slot] : &S.full[slot], ph, kDWaitLimit) || *(volatile int*)&S.abort) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t xa = tc::smem_u32(S.x[slot]), xb = xa + (uint32_t)a_bytes;
#pragma unroll
                for (int j = 0; j < kTK / kDStepK; ++j) {
                    const uint32_t ko = (uint32_t)(j * kDStepK * 4);     // 32 bytes per K = 8 step
                    const uint64_t ah = tc::smem_desc_sw64(xa + ko), bh = tc::smem_desc_sw64(xb + ko);
                    tc::mma_tf32(tmem, ah, bh, idesc, (s | j) ? 1u : 0u);
                    if (SPLIT) {
                        const uint32_t la = tc::smem_u32(S.lo[slot]), lb = la + (uint32_t)a_bytes;
                        tc::mma_tf32(tmem, ah, tc::smem_desc_sw64(lb + ko), idesc, 1);
                        tc::mma_tf32(tmem, tc::smem_desc_sw64(la + ko), bh, idesc, 1);
                    }
                }
                tc::mma_commit(&S.empty[slot]);
            }
            if (!ok) {
                *(volatile int*)&S.abort = 1;
                atomicExch(D.err, 1);
            }
            tc::mma_commit(&S.done);
        }
    } else {
        // ---- converters (warps 2-5, split operands): lo = x - tf32(x) of every stage
        const int ct = threadIdx.x - 64;
        for (int s = 0; SPLIT && s < nstage; ++s) {
            const int slot = s % kTStages;
            const uint32_t ph = (uint32_t)(s / kTStages) & 1u;
            const bool ok = tc::mbar_wait(&S.full[slot], ph, kDWaitLimit) && !*(volatile int*)&S.abort;
            if (ok) {
                const float4* xs = reinterpret_cast<const float4*>(S.x[slot]);
                float4* ls = reinterpret_cast<float4*>(S.lo[slot]);
                const int n4 = (a_bytes + b_bytes) / 16;
                for (int i = ct; i < n4; i += 128) {
                    const float4 v = xs[i];
                    ls[i] = make_float4(v.x - to_tf32(v.x), v.y - to_tf32(v.y), v.z - to_tf32(v.z), v.w - to_tf32(v.w));
                }
            } else if (ct == 0) {
                *(volatile int*)&S.abort = 1;
                atomicExch(D.err, 1);
            }
            tc::fence_proxy_async();                          // the tensor cores read what was written
            tc::mbar_arrive(&S.conv[slot]);
            if (!ok) break;
        }
    }
    // ---- epilogue (warps 2-5): TMEM lane quadrant warp % 4 holds rows 32 (warp % 4) ..
    const bool epi = warp >= 2;
    bool fin = true;
    if (threadIdx.x == 64) fin = tc::mbar_wait(&S.done, 0, kDWaitLimit);
    if (threadIdx.x == 64 && !fin) atomicExch(D.err, 1);
    __syncthreads();                                         // also: every stage is idle now
    tc::fence_after_sync();
    float* T = reinterpret_cast<float*>(S.x[0]);
    constexpr int kTS = kDEpiCols + 1;
    float* Cb = D.C + (int64_t)b * D.n * D.n;
    const int q = warp & 3, et = threadIdx.x - 64;
    for (int c0 = 0; c0 < NT; c0 += kDEpiCols) {
        const int cw = min(kDEpiCols, NT - c0);
        if (epi) {
            for (int c = 0; c < cw; c += 16) {
                float v[16];
                tc::tmem_ld16(tmem + (uint32_t)(c0 + c) + ((uint32_t)(32 * q) << 16), v);
#pragma unroll
                for (int x = 0; x < 16; ++x) T[(32 * q + lane) * kTS + c + x] = v[x];
            }
        }
        __syncthreads();
        if (epi) {
            const int col0 = tn * NT + c0;
            const int ncol = min(cw, D.n - col0);
            for (int r = et >> 5; r < kDM; r += 4) {
                const int row = tm * kDM + r;
                if (row >= D.n) break;
                float* out = Cb + (int64_t)row * D.n + col0;
                for (int c = lane; c < ncol; c += 32) {
                    const float v = D.alpha * T[r * kTS + c];
                    out[c] = D.beta == 0.f ? v : v + D.beta * out[c];
                }
            }
        }
        __syncthreads();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kDNMax);
    }
}

// B^T of every matrix of a batch (32 x 32 tiles through shared memory).
__global__ void k_dense_transpose(int64_t nb, int n, const float* __restrict__ B, float* __restrict__ Bt) {
    __shared__ float t[32][33];
    const int tiles = (n + 31) / 32;
    const int64_t total = nb * tiles * tiles;
    for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
        const int64_t m = w / ((int64_t)tiles * tiles);
        const int rest = (int)(w - m * tiles * tiles);
        const int ti = rest / tiles, tj = rest - ti * tiles;
        const float* src = B + m * n * n;
        float* dst = Bt + m * n * n;
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int i = ti * 32 + r, j = tj * 32 + threadIdx.x;
            t[r][threadIdx.x] = (i < n && j < n) ? src[(int64_t)i * n + j] : 0.f;
        }
        __syncthreads();
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int j = tj * 32 + r, i = ti * 32 + threadIdx.x;
            if (i < n && j < n) dst[(int64_t)j * n + i] = t[threadIdx.x][r];
        }
        __syncthreads();
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

namespace {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        DBG_CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !p) fail(DBCSR_ECUDA, "dense_gemm: cuTensorMapEncodeTiled not found");
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tensor map over a batch of n x n row-major FP32 matrices: boxes of 16 columns x rows rows of
// one matrix, 64-byte swizzled (n a multiple of 4: row strides of whole 16-byte units).
CUtensorMap batch_map(const float* base, int n, int64_t nb, int rows) {
    CUtensorMap m;
    const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)nb};
    const cuuint64_t strides[2] = {(cuuint64_t)n * 4, (cuuint64_t)n * n * 4};
    const cuuint32_t box[3] = {(cuuint32_t)kTK, (cuuint32_t)rows, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = tensor_map_encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims,
                                            strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                            CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(DBCSR_ECUDA, "dense_gemm: cuTensorMapEncodeTiled failed");
    return m;
}

}  // namespace

void dense_gemm_tf32(int64_t nb, int n, float alpha, const float* A, const float* B, float beta, float* C, bool split,
                     cudaStream_t s) {
    if (nb <= 0 || n <= 0) return;
    if (nb > 65535) fail(DBCSR_ECAPACITY, "dense_gemm: more than 65535 matrices in one batch");
    const bool aligned = (reinterpret_cast<uintptr_t>(A) & 15) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;
    if (n % 4 == 0 && aligned) {
        // operands straight from the matrices: A by rows, B^T (one transpose pass) by rows
        const int ntm = (int)ceil_div(n, kDM);
        const int ntn = (int)ceil_div(n, kDNMax);
        const int NT = (int)ceil_div(ceil_div(n, ntn), 16) * 16;
        DBuf<float> bt;
        DBuf<int> err;
        bt.alloc(nb * n * (int64_t)n, s);
        err.alloc(1, s);
        err.zero();
        const int64_t tiles = nb * ceil_div(n, 32) * ceil_div(n, 32);
        k_dense_transpose<<<grid_for(tiles, 1), dim3(32, 8), 0, s>>>(nb, n, B, bt.p);
        DBG_LAUNCH_CK();
        const CUtensorMap ma = batch_map(A, n, nb, kDM), mb = batch_map(bt.p, n, nb, NT);
        const TmaArgs d{n, ntm, ntn, NT, alpha, beta, C, err.p};
        const dim3 grid((unsigned)ntm, (unsigned)ntn, (unsigned)nb);
        if (split) {
            const size_t sm = sizeof(TmaShared<true>) + 1024;
            allow_dyn_smem(k_dense_tf32_tma<true>, sm);
            k_dense_tf32_tma<true><<<grid, kTThreads, sm, s>>>(ma, mb, d);
        } else {
            const size_t sm = sizeof(TmaShared<false>) + 1024;
            allow_dyn_smem(k_dense_tf32_tma<false>, sm);
            k_dense_tf32_tma<false><<<grid, kTThreads, sm, s>>>(ma, mb, d);
        }
        DBG_LAUNCH_CK();
        int e = 0;
        DBG_CK(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        DBG_CK(cudaStreamSynchronize(s));
        if (e) fail(DBCSR_ETIMEOUT, "dense_gemm: a wait of the tensor-core kernel ran out");
        return;
    }
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
