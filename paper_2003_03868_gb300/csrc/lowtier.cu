// The low-precision tier of the block-sparse product on the 5th-generation tensor cores
// (tcgen05.mma with FP32 accumulators in tensor memory): split-BF16 (x = hi + lo, three
// products hi*hi + hi*lo + lo*hi) or plain BF16 operands.  The paper runs small-matrix
// kernels per block triple and names low precision for these low-intensity products
// (sections "Batched execution" and "Outlook" / approximate computing); atom blocks of
// 5 to 23 rows fill only a small part of a tensor-core tile, so here the products run on
// groups of neighbouring atom blocks instead:
//
//   * groups: the block rows (= columns) are partitioned into groups of at most
//     kGroupWidth rows (kGroupMembers blocks) by merging blocks along the strongest
//     couplings of a matrix (single linkage on the block norms, width-capped).  For water
//     that gathers a few neighbouring molecules into one group;
//   * tiles: the product's operands and result are read as dense group tiles (zeros where
//     a group tile holds no atom block); C tile (G, G') = sum over G'' of A(G, G'') B(G'', G');
//   * the C tiles are those holding at least one atom block the product forms (after the
//     atom-level prescreen of the caller), and the epilogue writes exactly those atom
//     blocks, with their FP64 norms and distances to 1.  The result is the atom-level
//     product: a group tile only adds zero terms.
//
// Operands are packed once per product into the K-major no-swizzle layout of the tensor
// cores (tc05.cuh), 128 rows per tile, K in steps of 16: per step and part (hi, lo) two
// chunks of 128 x 8 BF16.  One CTA per SM runs a persistent loop over C tiles with
// specialised warps: warp 0 streams the A and B steps of the tile's stack into a ring of
// shared-memory stages with bulk copies, warp 1 issues the MMAs (M = 128, N = the column
// group's width rounded up to 16, K = 16) into one of two TMEM accumulators, and warps 2-5
// read the finished accumulator back and write the atom blocks.  Every wait is bounded: a
// wait that runs out sets an error flag and the kernel winds down.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "tc05.cuh"

namespace dbg {

namespace {

constexpr int kTileRows = 128;                 // M of the MMA; rows of every packed tile
constexpr int kStageBytesMax = 2 * 2 * 2 * kTileRows * 16;   // A and B steps, hi and lo: 16 KB
constexpr int kStages = 10;
constexpr int kLtThreads = 192;                // producer, MMA, 4 epilogue warps
constexpr int kTmemCols = 256;                 // two accumulators of up to 128 columns
constexpr long long kWaitLimit = 4000000000ll; // about 2 s at 2 GHz

// ------------------------------------------------------------------ groups (host)
struct Dsu {
    std::vector<int32_t> p, w, n;
    int32_t find(int32_t x) {
        while (p[x] != x) {
            p[x] = p[p[x]];
            x = p[x];
        }
        return x;
    }
};

}  // namespace

std::shared_ptr<Groups> build_groups(dbcsr_matrix_* M) {
    check_finalized(M);
    ensure_norms(M);
    cudaStream_t s = M->stream;
    const int32_t nb = M->nblk;
    std::vector<int64_t> rp(nb + 1);
    std::vector<int32_t> col(std::max<int64_t>(M->nnzb, 1));
    std::vector<double> nrm(std::max<int64_t>(M->nnzb, 1));
    DBG_CK(cudaMemcpyAsync(rp.data(), M->rp.p, sizeof(int64_t) * (nb + 1), cudaMemcpyDeviceToHost, s));
    if (M->nnzb) {
        DBG_CK(cudaMemcpyAsync(col.data(), M->col.p, sizeof(int32_t) * M->nnzb, cudaMemcpyDeviceToHost, s));
        DBG_CK(cudaMemcpyAsync(nrm.data(), M->norms.p, sizeof(double) * M->nnzb, cudaMemcpyDeviceToHost, s));
    }
    DBG_CK(cudaStreamSynchronize(s));
    // candidate merges: the kTop strongest off-diagonal couplings of every block row
    constexpr int kTop = 12;
    struct Edge {
        double w;
        int32_t a, b;
    };
    std::vector<Edge> edges;
    edges.reserve((size_t)nb * kTop);
    std::vector<std::pair<double, int32_t>> row;
    for (int32_t i = 0; i < nb; ++i) {
        row.clear();
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
            if (col[q] != i) row.push_back({nrm[q], col[q]});
        const size_t t = std::min<size_t>(kTop, row.size());
        std::partial_sort(row.begin(), row.begin() + t, row.end(), [](const auto& x, const auto& y) {
            return x.first > y.first || (x.first == y.first && x.second < y.second);
        });
        for (size_t e = 0; e < t; ++e)
            edges.push_back({row[e].first, std::min(i, row[e].second), std::max(i, row[e].second)});
    }
    std::sort(edges.begin(), edges.end(), [](const Edge& x, const Edge& y) {
        if (x.w != y.w) return x.w > y.w;
        if (x.a != y.a) return x.a < y.a;
        return x.b < y.b;
    });
    Dsu d;
    d.p.resize(nb);
    d.w.resize(nb);
    d.n.assign(nb, 1);
    std::iota(d.p.begin(), d.p.end(), 0);
    for (int32_t i = 0; i < nb; ++i) d.w[i] = M->h_bs[i];
    for (const Edge& e : edges) {
        int32_t a = d.find(e.a), b = d.find(e.b);
        if (a == b || d.w[a] + d.w[b] > kGroupWidth || d.n[a] + d.n[b] > kGroupMembers) continue;
        if (b < a) std::swap(a, b);
        d.p[b] = a;
        d.w[a] += d.w[b];
        d.n[a] += d.n[b];
    }
    // groups numbered by their first block; members in ascending block order
    auto g = std::make_shared<Groups>();
    std::vector<int32_t> gid(nb, -1), g_of(nb), g_pos(nb), g_ptr, g_mem(nb), g_w;
    int32_t ng = 0;
    for (int32_t i = 0; i < nb; ++i) {
        const int32_t r = d.find(i);
        if (gid[r] < 0) gid[r] = ng++;
        g_of[i] = gid[r];
    }
    g_ptr.assign(ng + 1, 0);
    g_w.assign(ng, 0);
    for (int32_t i = 0; i < nb; ++i) g_ptr[g_of[i] + 1]++;
    for (int32_t k = 0; k < ng; ++k) g_ptr[k + 1] += g_ptr[k];
    std::vector<int32_t> fill(g_ptr.begin(), g_ptr.end() - 1);
    int max_members = 0;
    for (int32_t i = 0; i < nb; ++i) {
        const int32_t k = g_of[i];
        g_mem[fill[k]++] = i;
        g_pos[i] = g_w[k];
        g_w[k] += M->h_bs[i];
    }
    for (int32_t k = 0; k < ng; ++k) max_members = std::max(max_members, g_ptr[k + 1] - g_ptr[k]);
    g->ngrp = ng;
    g->nblk = nb;
    g->max_members = max_members;
    g->h_w = g_w;
    g->g_of.alloc(nb, s);
    g->g_pos.alloc(nb, s);
    g->g_ptr.alloc(ng + 1, s);
    g->g_mem.alloc(nb, s);
    g->g_w.alloc(ng, s);
    DBG_CK(cudaMemcpyAsync(g->g_of.p, g_of.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s));
    DBG_CK(cudaMemcpyAsync(g->g_pos.p, g_pos.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s));
    DBG_CK(cudaMemcpyAsync(g->g_ptr.p, g_ptr.data(), sizeof(int32_t) * (ng + 1), cudaMemcpyHostToDevice, s));
    DBG_CK(cudaMemcpyAsync(g->g_mem.p, g_mem.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s));
    DBG_CK(cudaMemcpyAsync(g->g_w.p, g_w.data(), sizeof(int32_t) * ng, cudaMemcpyHostToDevice, s));
    DBG_CK(cudaStreamSynchronize(s));           // the host vectors go out of scope
    return g;
}

namespace {

// ------------------------------------------------------------------ group tile patterns
__device__ int lt_block_scan(int v, int* sh, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sh[lane] = t;
    }
    __syncthreads();
    const int excl = (warp ? sh[warp - 1] : 0) + x - v;
    total = sh[nw - 1];
    __syncthreads();
    return excl;
}

__device__ __forceinline__ int lt_rank(const uint32_t* bm, const int* wpre, int32_t g) {
    return wpre[g >> 5] + __popc(bm[g >> 5] & ((1u << (g & 31)) - 1u));
}

struct GView {
    const int32_t* g_of; const int32_t* g_pos; const int32_t* g_ptr; const int32_t* g_mem; const int32_t* g_w;
};

// Bitmap (and prefix popcounts) of the groups reached by the blocks of group row G of a
// block pattern (rp, col); use[q] (nullable) selects blocks.  Returns the number of groups.
__device__ int lt_group_row(const GView& g, int32_t G, const int64_t* rp, const int32_t* col, const uint8_t* use,
                            uint32_t* bm, int* wpre, int nwords, int* sh) {
    for (int w = threadIdx.x; w < nwords; w += blockDim.x) bm[w] = 0u;
    __syncthreads();
    for (int32_t m = g.g_ptr[G]; m < g.g_ptr[G + 1]; ++m) {
        const int32_t I = g.g_mem[m];
        for (int64_t q = rp[I] + threadIdx.x; q < rp[I + 1]; q += blockDim.x)
            if (!use || use[q]) {
                const int32_t c = g.g_of[col[q]];
                atomicOr(&bm[c >> 5], 1u << (c & 31));
            }
    }
    __syncthreads();
    const int per = (nwords + blockDim.x - 1) / blockDim.x;
    const int lo = min(nwords, (int)threadIdx.x * per), hi = min(nwords, lo + per);
    int s = 0;
    for (int w = lo; w < hi; ++w) s += __popc(bm[w]);
    int total;
    int run = lt_block_scan(s, sh, total);
    for (int w = lo; w < hi; ++w) {
        wpre[w] = run;
        run += __popc(bm[w]);
    }
    __syncthreads();
    return total;
}

// fill == 0: cnt[G] = number of tiles of group row G.  fill == 1: tile rows/columns and the
// tile of every selected block (blk_tile[q], -1 for blocks not selected).
__global__ void k_gt_pattern(int32_t ngrp, GView g, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const uint8_t* __restrict__ use, int nwords, int fill, int64_t* __restrict__ cnt,
                             const int64_t* __restrict__ t_rp, int32_t* __restrict__ t_row,
                             int32_t* __restrict__ t_col, int32_t* __restrict__ blk_tile) {
    extern __shared__ uint32_t lt_smem[];
    __shared__ int sh[32];
    uint32_t* bm = lt_smem;
    int* wpre = (int*)(lt_smem + nwords);
    for (int32_t G = blockIdx.x; G < ngrp; G += gridDim.x) {
        const int n = lt_group_row(g, G, rp, col, use, bm, wpre, nwords, sh);
        if (!fill) {
            if (threadIdx.x == 0) cnt[G] = n;
        } else {
            const int64_t base = t_rp[G];
            for (int w = threadIdx.x; w < nwords; w += blockDim.x) {
                uint32_t bits = bm[w];
                int r = wpre[w];
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    t_row[base + r] = G;
                    t_col[base + r] = w * 32 + b;
                    ++r;
                }
            }
            if (blk_tile)
                for (int32_t m = g.g_ptr[G]; m < g.g_ptr[G + 1]; ++m) {
                    const int32_t I = g.g_mem[m];
                    for (int64_t q = rp[I] + threadIdx.x; q < rp[I + 1]; q += blockDim.x)
                        blk_tile[q] = (!use || use[q]) ? (int32_t)(base + lt_rank(bm, wpre, g.g_of[col[q]])) : -1;
                }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int lt_ksteps(int w) { return (w + 15) >> 4; }

// Packed bytes of every tile: ceil(width of its K group / 16) steps of nparts * 4 KB.
__global__ void k_gt_bytes(int64_t nt, const int32_t* __restrict__ t_kgrp, const int32_t* __restrict__ g_w,
                           int nparts, int64_t* __restrict__ bytes) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x)
        bytes[t] = (int64_t)lt_ksteps(g_w[t_kgrp[t]]) * nparts * 2 * kTileRows * 16;
}

// For a symmetric pattern: tT[t] = the tile (c, r) of tile t = (r, c).
__global__ void k_gt_transpose(int64_t nt, const int32_t* __restrict__ t_row, const int32_t* __restrict__ t_col,
                               const int64_t* __restrict__ t_rp, int32_t* __restrict__ tT, int* __restrict__ err) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = t_row[t], c = t_col[t];
        int64_t lo = t_rp[c], hi = t_rp[c + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (t_col[mid] < r) lo = mid + 1; else hi = mid;
        }
        const bool ok = lo < t_rp[c + 1] && t_col[lo] == r;
        tT[t] = ok ? (int32_t)lo : -1;
        if (!ok) atomicExch(err, 2);
    }
}

// ------------------------------------------------------------------ packing
// FP64 -> BF16, round to nearest even, from the IEEE-754 encodings (binary32 range; values
// below its normal range become signed zero).
__device__ __forceinline__ uint16_t lt_bf16_bits(double x) {
    const uint64_t u = (uint64_t)__double_as_longlong(x);
    const uint16_t sign = (uint16_t)((u >> 48) & 0x8000u);
    const int e = (int)((u >> 52) & 0x7ff);
    if (e == 0x7ff) return (uint16_t)(sign | 0x7f80u | ((u & 0xfffffffffffffull) ? 0x40u : 0u));
    const int eb = e - 1023 + 127;               // biased binary32 exponent
    if (eb < 1) return sign;                     // below the normal range
    uint64_t mant = u & 0xfffffffffffffull;      // 52 bits; keep 7
    const uint64_t keep = mant >> 45, rest = mant & ((1ull << 45) - 1);
    const uint64_t half = 1ull << 44;
    uint32_t m7 = (uint32_t)keep;
    int ex = eb;
    if (rest > half || (rest == half && (m7 & 1u))) {
        if (++m7 == 128u) {
            m7 = 0;
            ++ex;
        }
    }
    if (ex >= 255) return (uint16_t)(sign | 0x7f80u);
    return (uint16_t)(sign | ((uint32_t)ex << 7) | m7);
}
__device__ __forceinline__ double lt_bf16_value(uint16_t b) {
    return (double)__uint_as_float((uint32_t)b << 16);
}

struct PackArgs {
    int64_t nb;
    const int32_t* row; const int32_t* col; const int64_t* off; const double* data; const int32_t* bs;
    const int32_t* blk_tile; const int64_t* t_off;
    const int32_t* g_pos;
    int transpose;       // 0: block (I, K) -> rows of I, K columns of K; 1: block (K, J) -> rows of J, K of K
    int nparts;          // 1: plain BF16; 2: hi and lo
    uint8_t* pack;
};

// One warp per block: its elements into the tile, at (row, kcol) -> step kcol / 16, chunk
// (kcol / 8) % 2, row, element kcol % 8; the lo part one chunk pair after the hi part.
__global__ void k_gt_pack(PackArgs P) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < P.nb; b += warps) {
        const int32_t t = P.blk_tile[b];
        if (t < 0) continue;
        const int32_t I = P.row[b], J = P.col[b];
        const int m = P.bs[I], n = P.bs[J];
        const int pi = P.g_pos[I], pj = P.g_pos[J];
        const double* src = P.data + P.off[b];
        uint8_t* base = P.pack + P.t_off[t];
        const int slab = P.nparts * 2 * kTileRows * 16;
        for (int e = lane; e < m * n; e += 32) {
            const int i = e / n, j = e - i * n;
            const int r = P.transpose ? pj + j : pi + i;
            const int kc = P.transpose ? pi + i : pj + j;
            const double x = src[e];
            const uint16_t hi = lt_bf16_bits(x);
            uint8_t* p = base + (int64_t)(kc >> 4) * slab + ((kc >> 3) & 1) * (kTileRows * 16) + r * 16 + (kc & 7) * 2;
            *(uint16_t*)p = hi;
            if (P.nparts == 2) *(uint16_t*)(p + 2 * kTileRows * 16) = lt_bf16_bits(x - lt_bf16_value(hi));
        }
    }
}

// ------------------------------------------------------------------ product stacks
struct StackArgs {
    GView g;
    const int64_t* c_trp; const int32_t* c_tcol;          // C tiles by group row
    const int64_t* a_trp; const int32_t* a_tcol;          // A tiles by group row (A-style)
    const int64_t* b_trp; const int32_t* b_tcol;          // B tiles by K group row
    const int32_t* b_map;                                 // B operand tile -> packed tile (nullable)
    int64_t* cnt;                                         // count pass: entries per C tile (global)
    const int64_t* s_ptr;                                 // fill pass: stack start of each C tile
    int32_t* st_a; int32_t* st_b;
    int32_t* cursor;                                      // global cursors (when not in shared memory)
    int fill, use_smem;
};

// Per group row G: for every A tile (G, G'') in ascending G'' and every B tile (G'', G')
// whose C tile (G, G') exists, one stack entry of that C tile.  Entries of a C tile are in
// ascending G''.
__global__ void k_gt_stack(int32_t ngrp, StackArgs S, int nwords) {
    extern __shared__ uint32_t lt_smem[];
    __shared__ int sh[32];
    uint32_t* bm = lt_smem;
    int* wpre = (int*)(lt_smem + nwords);
    int32_t* cur = (int32_t*)(wpre + nwords);
    for (int32_t G = blockIdx.x; G < ngrp; G += gridDim.x) {
        for (int w = threadIdx.x; w < nwords; w += blockDim.x) bm[w] = 0u;
        __syncthreads();
        const int64_t c0 = S.c_trp[G], c1 = S.c_trp[G + 1];
        for (int64_t t = c0 + threadIdx.x; t < c1; t += blockDim.x) {
            const int32_t c = S.c_tcol[t];
            atomicOr(&bm[c >> 5], 1u << (c & 31));
        }
        __syncthreads();
        {
            const int per = (nwords + blockDim.x - 1) / blockDim.x;
            const int lo = min(nwords, (int)threadIdx.x * per), hi = min(nwords, lo + per);
            int s = 0;
            for (int w = lo; w < hi; ++w) s += __popc(bm[w]);
            int total;
            int run = lt_block_scan(s, sh, total);
            for (int w = lo; w < hi; ++w) {
                wpre[w] = run;
                run += __popc(bm[w]);
            }
        }
        const int nct = (int)(c1 - c0);
        int32_t* cc = S.use_smem ? cur : S.cursor + c0;
        for (int r = threadIdx.x; r < nct; r += blockDim.x) cc[r] = 0;
        __syncthreads();
        for (int64_t ta = S.a_trp[G]; ta < S.a_trp[G + 1]; ++ta) {
            const int32_t K = S.a_tcol[ta];
            for (int64_t tb = S.b_trp[K] + threadIdx.x; tb < S.b_trp[K + 1]; tb += blockDim.x) {
                const int32_t c = S.b_tcol[tb];
                if (!(bm[c >> 5] & (1u << (c & 31)))) continue;
                // a B tile without its transposed twin (an asymmetric pattern declared symmetric) is
                // left out; the k_gt_transpose error flag reports it
                const int32_t bt = S.b_map ? S.b_map[tb] : (int32_t)tb;
                if (bt < 0) continue;
                const int r = lt_rank(bm, wpre, c);
                const int32_t at = cc[r];
                cc[r] = at + 1;
                if (S.fill) {
                    const int64_t pos = S.s_ptr[c0 + r] + at;
                    S.st_a[pos] = (int32_t)ta;
                    S.st_b[pos] = bt;
                }
            }
            __syncthreads();
        }
        if (!S.fill)
            for (int r = threadIdx.x; r < nct; r += blockDim.x) S.cnt[c0 + r] = cc[r];
        __syncthreads();
    }
}

// ------------------------------------------------------------------ the tensor-core kernel
struct LtArgs {
    int64_t ntiles;
    const int32_t* c_trow; const int32_t* c_tcol; const int64_t* s_ptr;
    const int32_t* st_a; const int32_t* st_b;
    const int32_t* a_tkgrp;                  // K group of every A tile
    const uint8_t* a_pack; const int64_t* a_off;
    const uint8_t* b_pack; const int64_t* b_off;
    GView g;
    const int32_t* bs;
    const int64_t* f_rp; const int32_t* f_col; const uint8_t* f_comp; const int64_t* f_off; const int64_t* f_cin;
    const int64_t* ci_off; const double* ci_data;
    double alpha, beta;
    double* c_data; double* c_norm; double* c_dev2;
    int nparts;
    int* err;                                // 1: a wait ran out
};

struct LtShared {
    alignas(1024) uint8_t stage[kStages][kStageBytesMax];
    double psq[kGroupMembers][kTileRows];    // per (column member, row): sum of squares
    double pd2[kTileRows];                   // per row: squared distance to 1 of the diagonal block
    int32_t tbl[kGroupMembers][kGroupMembers];
    int16_t rowm[kTileRows];                 // member | (row within member) << 5, -1 beyond the width
    int16_t colm[kTileRows];
    int32_t rowblk[kGroupMembers];
    int32_t colblk[kGroupMembers];
    uint64_t full[kStages], empty[kStages], acc_full[2], acc_empty[2], fin;
    uint32_t tmem_base;
    int abort;                               // set once by a role whose wait ran out
    int epi_stop;                            // the epilogue's snapshot of abort
};

__device__ __forceinline__ void lt_epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ __forceinline__ int lt_aborted(const LtShared& S) { return *(volatile const int*)&S.abort; }

__device__ __forceinline__ void lt_fail(const LtArgs& A, LtShared& S) {
    *(volatile int*)&S.abort = 1;
    atomicExch(A.err, 1);
}

__global__ void __launch_bounds__(kLtThreads, 1) k_lowtier(LtArgs A) {
    extern __shared__ __align__(1024) uint8_t lt_dyn[];
    LtShared& S = *reinterpret_cast<LtShared*>((reinterpret_cast<uintptr_t>(lt_dyn) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            tc::mbar_init(&S.full[i], 1);
            tc::mbar_init(&S.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&S.acc_full[i], 1);
            tc::mbar_init(&S.acc_empty[i], 128);
        }
        tc::mbar_init(&S.fin, 1);
        S.abort = 0;
        S.epi_stop = 0;
        tc::fence_barrier_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(&S.tmem_base, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = S.tmem_base;
    const int slab = A.nparts * 2 * kTileRows * 16;   // bytes of one K step of one operand

    if (warp == 0) {
        // ---------------- producer: the tile's stack, K step by K step, into the stage ring
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int64_t armed = 0;
            for (int64_t t = blockIdx.x; t < A.ntiles && !lt_aborted(S); t += gridDim.x) {
                for (int64_t e = A.s_ptr[t]; e < A.s_ptr[t + 1] && !lt_aborted(S); ++e) {
                    const int32_t ta = A.st_a[e], tb = A.st_b[e];
                    const int ks = lt_ksteps(A.g.g_w[A.a_tkgrp[ta]]);
                    const uint8_t* pa = A.a_pack + A.a_off[ta];
                    const uint8_t* pb = A.b_pack + A.b_off[tb];
                    for (int k = 0; k < ks; ++k) {
                        if (!tc::mbar_wait(&S.empty[stage], phase ^ 1u, kWaitLimit)) {
                            lt_fail(A, S);
                            break;
                        }
                        tc::mbar_arrive_expect_tx(&S.full[stage], 2 * slab);
                        tc::bulk_g2s(S.stage[stage], pa + (int64_t)k * slab, slab, &S.full[stage]);
                        tc::bulk_g2s(S.stage[stage] + slab, pb + (int64_t)k * slab, slab, &S.full[stage]);
                        ++armed;
                        if (++stage == kStages) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
            }
            // no copy may still be landing in shared memory when the CTA exits: wait (bounded)
            // for the last armed stages (after a normal run the MMA warp consumed them all)
            for (int64_t x = 0; x < armed && x < kStages; ++x) {
                if (--stage < 0) {
                    stage = kStages - 1;
                    phase ^= 1u;
                }
                if (!tc::mbar_wait(&S.full[stage], phase, kWaitLimit)) lt_fail(A, S);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int it = 0;
            for (int64_t t = blockIdx.x; t < A.ntiles && !lt_aborted(S); t += gridDim.x, ++it) {
                const int acc = it & 1;
                const uint32_t acc_phase = (uint32_t)(it >> 1) & 1u;
                if (!tc::mbar_wait(&S.acc_empty[acc], acc_phase ^ 1u, kWaitLimit)) {
                    lt_fail(A, S);
                    break;
                }
                tc::fence_after_sync();
                const int N = ((A.g.g_w[A.c_tcol[t]] + 15) >> 4) << 4;
                const uint32_t idesc = tc::instr_desc(1, kTileRows, N);
                const uint32_t d_tmem = tmem + (uint32_t)(acc * 128);
                uint32_t accumulate = 0;
                for (int64_t e = A.s_ptr[t]; e < A.s_ptr[t + 1] && !lt_aborted(S); ++e) {
                    const int ks = lt_ksteps(A.g.g_w[A.a_tkgrp[A.st_a[e]]]);
                    for (int k = 0; k < ks; ++k) {
                        if (!tc::mbar_wait(&S.full[stage], phase, kWaitLimit)) {
                            lt_fail(A, S);
                            break;
                        }
                        tc::fence_after_sync();
                        const uint32_t sa = tc::smem_u32(S.stage[stage]);
                        const uint32_t sb = sa + (uint32_t)slab;
                        const uint32_t part = 2 * kTileRows * 16;   // hi -> lo
                        const uint64_t ah = tc::smem_desc(sa, kTileRows * 16, 128);
                        const uint64_t bh = tc::smem_desc(sb, kTileRows * 16, 128);
                        tc::mma_f16(d_tmem, ah, bh, idesc, accumulate);
                        accumulate = 1;
                        if (A.nparts == 2) {
                            const uint64_t al = tc::smem_desc(sa + part, kTileRows * 16, 128);
                            const uint64_t bl = tc::smem_desc(sb + part, kTileRows * 16, 128);
                            tc::mma_f16(d_tmem, ah, bl, idesc, 1);
                            tc::mma_f16(d_tmem, al, bh, idesc, 1);
                        }
                        tc::mma_commit(&S.empty[stage]);         // the stage is free once these MMAs ran
                        if (++stage == kStages) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
                tc::mma_commit(&S.acc_full[acc]);                // the accumulator is complete
            }
            // every MMA this thread issued has completed before the TMEM is released
            tc::mma_commit(&S.fin);
            if (!tc::mbar_wait(&S.fin, 0, kWaitLimit)) lt_fail(A, S);
        }
    } else {
        // ---------------- epilogue: warps 2..5, TMEM lanes 32 * (warp % 4) ..
        const int et = threadIdx.x - 64;                          // 0..127
        const int q = warp & 3;
        const int r = 32 * q + lane;                              // tile row of this thread
        int it = 0;
        for (int64_t t = blockIdx.x; t < A.ntiles; t += gridDim.x, ++it) {
            if (et == 0) S.epi_stop = lt_aborted(S);
            lt_epi_sync();
            if (S.epi_stop) break;
            const int acc = it & 1;
            const uint32_t acc_phase = (uint32_t)(it >> 1) & 1u;
            const int32_t G = A.c_trow[t], Gc = A.c_tcol[t];
            const int32_t m0 = A.g.g_ptr[G], nm = A.g.g_ptr[G + 1] - m0;
            const int32_t n0 = A.g.g_ptr[Gc], nn = A.g.g_ptr[Gc + 1] - n0;
            const int wr = A.g.g_w[G], wc = A.g.g_w[Gc];
            // the atom blocks of the tile this product writes: tbl[a][b] = formed block or -1
            for (int p = et; p < nm * nn; p += 128) {
                const int a = p / nn, b = p - a * nn;
                const int32_t I = A.g.g_mem[m0 + a], J = A.g.g_mem[n0 + b];
                int64_t lo = A.f_rp[I], hi = A.f_rp[I + 1];
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (A.f_col[mid] < J) lo = mid + 1; else hi = mid;
                }
                const bool found = lo < A.f_rp[I + 1] && A.f_col[lo] == J && A.f_comp[lo];
                S.tbl[a][b] = found ? (int32_t)lo : -1;
            }
            if (et < nm) S.rowblk[et] = A.g.g_mem[m0 + et];
            if (et < nn) S.colblk[et] = A.g.g_mem[n0 + et];
            for (int a = et; a < kTileRows; a += 128) S.rowm[a] = -1;
            for (int a = et; a < kTileRows; a += 128) S.colm[a] = -1;
            lt_epi_sync();
            if (et < nm) {
                const int32_t I = S.rowblk[et];
                const int p0 = A.g.g_pos[I];
                for (int i = 0; i < A.bs[I]; ++i) S.rowm[p0 + i] = (int16_t)(et | (i << 5));
            }
            if (et < nn) {
                const int32_t J = S.colblk[et];
                const int p0 = A.g.g_pos[J];
                for (int j = 0; j < A.bs[J]; ++j) S.colm[p0 + j] = (int16_t)(et | (j << 5));
            }
            for (int b = 0; b < nn; ++b) S.psq[b][r] = 0.0;
            S.pd2[r] = 0.0;
            lt_epi_sync();
            // every tile's accumulator phase completes (a tile without products commits no MMA
            // and is written as zeros, but its phase is still waited for)
            const bool empty = A.s_ptr[t] == A.s_ptr[t + 1];
            // the TMEM loads are warp-collective: a warp reads only if all its lanes saw the phase
            const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&S.acc_full[acc], acc_phase, kWaitLimit));
            if (!ok) lt_fail(A, S);
            tc::fence_after_sync();
            const int rv = (ok && r < wr) ? S.rowm[r] : -1;
            const int a = rv >= 0 ? (rv & 31) : 0, i = rv >= 0 ? (rv >> 5) : 0;
            const int32_t I = S.rowblk[a];
            const int ncol = ((wc + 15) >> 4) << 4;
            double sq = 0.0, d2 = 0.0;
            int cur_b = -1;
            for (int c0 = 0; c0 < ncol; c0 += 16) {
                float v[16];
                if (!empty && ok) {
                    tc::tmem_ld16(tmem + (uint32_t)(acc * 128 + c0) + ((uint32_t)(32 * q) << 16), v);
                } else {
#pragma unroll
                    for (int x = 0; x < 16; ++x) v[x] = 0.f;
                }
                if (rv < 0) continue;
#pragma unroll
                for (int x = 0; x < 16; ++x) {
                    const int c = c0 + x;
                    const int cv = c < wc ? S.colm[c] : -1;
                    if (cv < 0) continue;
                    const int b = cv & 31, j = cv >> 5;
                    if (b != cur_b) {
                        if (cur_b >= 0) S.psq[cur_b][r] = sq;
                        sq = 0.0;
                        cur_b = b;
                    }
                    const int64_t k = S.tbl[a][b];
                    if (k < 0) continue;
                    const int32_t J = S.colblk[b];
                    const int n = A.bs[J];
                    double val = A.alpha * (double)v[x];
                    const int64_t ci = A.f_cin ? A.f_cin[k] : -1;
                    if (ci >= 0) val = val + A.beta * A.ci_data[A.ci_off[ci] + (int64_t)i * n + j];
                    A.c_data[A.f_off[k] + (int64_t)i * n + j] = val;
                    sq = fma(val, val, sq);
                    if (I == J) {
                        const double w = (i == j) ? val - 1.0 : val;
                        d2 = fma(w, w, d2);
                    }
                }
            }
            if (cur_b >= 0) S.psq[cur_b][r] = sq;
            S.pd2[r] = d2;
            // the accumulator may be reused once every lane has read it
            tc::fence_before_sync();
            lt_epi_sync();
            tc::mbar_arrive(&S.acc_empty[acc]);
            // norms and distances to 1 of the written blocks, rows summed in order
            for (int p = et; p < nm * nn && ok; p += 128) {
                const int aa = p / nn, bb = p - aa * nn;
                const int32_t k = S.tbl[aa][bb];
                if (k < 0) continue;
                const int32_t Ia = S.rowblk[aa], Jb = S.colblk[bb];
                const int p0 = A.g.g_pos[Ia];
                double s2 = 0.0, dd = 0.0;
                for (int x = 0; x < A.bs[Ia]; ++x) {
                    s2 += S.psq[bb][p0 + x];
                    dd += S.pd2[p0 + x];
                }
                A.c_norm[k] = sqrt(s2);
                A.c_dev2[k] = (Ia == Jb) ? dd : s2;
            }
            lt_epi_sync();
        }
    }
    // wind down: every role is done; MMAs issued are complete (the epilogue waited on them)
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

}  // namespace

// ------------------------------------------------------------------ host side
namespace {

struct TilePattern {
    int64_t nt = 0;
    DBuf<int64_t> t_rp;          // [ngrp + 1]
    DBuf<int32_t> t_row, t_col;  // [nt]
    DBuf<int32_t> blk_tile;      // [nnzb] tile of every block
};

int pattern_words(int32_t ngrp) { return (ngrp + 31) / 32; }

TilePattern tile_pattern(const Groups& g, const int64_t* rp, const int32_t* col, const uint8_t* use, int64_t nnzb,
                         bool want_blk, cudaStream_t s) {
    TilePattern P;
    const int nwords = pattern_words(g.ngrp);
    const size_t sm = (size_t)2 * ((nwords + 1) & ~1) * sizeof(uint32_t);
    GView gv{g.g_of.p, g.g_pos.p, g.g_ptr.p, g.g_mem.p, g.g_w.p};
    DBuf<int64_t> cnt;
    cnt.alloc(g.ngrp, s);
    P.t_rp.alloc(g.ngrp + 1, s);
    allow_dyn_smem(k_gt_pattern, sm);
    const unsigned grid = (unsigned)std::min<int64_t>(g.ngrp, (int64_t)num_sms() * 8);
    k_gt_pattern<<<grid, 256, sm, s>>>(g.ngrp, gv, rp, col, use, nwords, 0, cnt.p, nullptr, nullptr, nullptr,
                                       nullptr);
    DBG_LAUNCH_CK();
    scan_exclusive(cnt.p, P.t_rp.p, g.ngrp, s);
    P.nt = read_i64(P.t_rp.p + g.ngrp, s);
    P.t_row.alloc(std::max<int64_t>(P.nt, 1), s);
    P.t_col.alloc(std::max<int64_t>(P.nt, 1), s);
    if (want_blk) P.blk_tile.alloc(std::max<int64_t>(nnzb, 1), s);
    k_gt_pattern<<<grid, 256, sm, s>>>(g.ngrp, gv, rp, col, use, nwords, 1, nullptr, P.t_rp.p, P.t_row.p, P.t_col.p,
                                       want_blk ? P.blk_tile.p : nullptr);
    DBG_LAUNCH_CK();
    return P;
}

// Offsets of the packed tiles (bytes) and the total.
int64_t tile_offsets(const TilePattern& P, const int32_t* t_kgrp, const Groups& g, int nparts, DBuf<int64_t>& off,
                     cudaStream_t s) {
    DBuf<int64_t> bytes;
    bytes.alloc(std::max<int64_t>(P.nt, 1), s);
    off.alloc(P.nt + 1, s);
    if (P.nt) {
        k_gt_bytes<<<grid_for(P.nt, 256), 256, 0, s>>>(P.nt, t_kgrp, g.g_w.p, nparts, bytes.p);
        DBG_LAUNCH_CK();
    }
    scan_exclusive(bytes.p, off.p, P.nt, s);
    return read_i64(off.p + P.nt, s);
}

}  // namespace

struct LowTierPlan {
    int nparts = 2;
    int64_t ntiles = 0, nentries = 0;
    TilePattern ap, bp, cp;
    DBuf<int64_t> a_off, b_off, s_ptr;
    DBuf<int32_t> st_a, st_b, b_map;
    DBuf<uint8_t> a_pack, b_pack;
    int64_t a_bytes = 0, b_bytes = 0;
    bool b_is_a = false;          // B's operand tiles are read from A's pack
    bool b_from_a_style = false;  // B's operand tiles are read from B's own rows (symmetric B)
    DBuf<int> err;
    std::shared_ptr<Groups> groups;
};

void lowtier_plan_delete(LowTierPlan* p) { delete p; }

namespace {

void pack_operand(const dbcsr_matrix_* M, const TilePattern& P, const DBuf<int64_t>& off, int64_t bytes,
                  DBuf<uint8_t>& pack, const Groups& g, int transpose, int nparts, cudaStream_t s) {
    if (!bytes || !M->nnzb) return;
    DBG_CK(cudaMemsetAsync(pack.p, 0, (size_t)bytes, s));
    PackArgs pa{M->nnzb, M->row.p, M->col.p, M->off.p, M->data.p, M->bs.p, P.blk_tile.p, off.p, g.g_pos.p,
                transpose, nparts, pack.p};
    k_gt_pack<<<grid_for(M->nnzb, 8), 256, 0, s>>>(pa);
    DBG_LAUNCH_CK();
}

}  // namespace

std::unique_ptr<LowTierPlan, void (*)(LowTierPlan*)> lowtier_prepare(int prec, dbcsr_matrix_* A, dbcsr_matrix_* B,
                                                                     std::shared_ptr<Groups> groups, bool sym_operands,
                                                                     const int64_t* f_rp, const int32_t* f_col,
                                                                     const uint8_t* f_comp, cudaStream_t s) {
    std::unique_ptr<LowTierPlan, void (*)(LowTierPlan*)> L(new LowTierPlan(), lowtier_plan_delete);
    const Groups& g = *groups;
    L->groups = groups;
    L->nparts = prec == DBCSR_BF16X3 ? 2 : 1;
    if (g.ngrp > kMaxBlockRowsLt) fail(DBCSR_ECAPACITY, "multiply: too many groups for the tensor-core tier");
    // A: rows = A's group rows, K = its column groups
    L->ap = tile_pattern(g, A->rp.p, A->col.p, nullptr, A->nnzb, true, s);
    L->a_bytes = tile_offsets(L->ap, L->ap.t_col.p, g, L->nparts, L->a_off, s);
    // B: symmetric operands read their K-major tiles from the A-style tiles of the transposed
    // position; otherwise B is packed transposed (rows = its column group, K = its row group)
    L->b_is_a = sym_operands && B == A;
    L->b_from_a_style = sym_operands;
    L->err.alloc(1, s);
    L->err.zero();
    if (!L->b_is_a) {
        L->bp = tile_pattern(g, B->rp.p, B->col.p, nullptr, B->nnzb, true, s);
        L->b_bytes = tile_offsets(L->bp, sym_operands ? L->bp.t_col.p : L->bp.t_row.p, g, L->nparts, L->b_off, s);
    }
    const TilePattern& bpat = L->b_is_a ? L->ap : L->bp;
    if (sym_operands && bpat.nt) {
        L->b_map.alloc(bpat.nt, s);
        k_gt_transpose<<<grid_for(bpat.nt, 256), 256, 0, s>>>(bpat.nt, bpat.t_row.p, bpat.t_col.p, bpat.t_rp.p,
                                                               L->b_map.p, L->err.p);
        DBG_LAUNCH_CK();
    }
    // C tiles: group pairs of the atom blocks the product computes
    const int32_t nblk = A->nblk;
    (void)nblk;
    L->cp = tile_pattern(g, f_rp, f_col, f_comp, 0, false, s);
    L->ntiles = L->cp.nt;
    // stacks
    const int nwords = pattern_words(g.ngrp);
    int64_t max_row = 0;
    {
        std::vector<int64_t> h(g.ngrp + 1);
        DBG_CK(cudaMemcpyAsync(h.data(), L->cp.t_rp.p, sizeof(int64_t) * (g.ngrp + 1), cudaMemcpyDeviceToHost, s));
        DBG_CK(cudaStreamSynchronize(s));
        for (int32_t k = 0; k < g.ngrp; ++k) max_row = std::max(max_row, h[k + 1] - h[k]);
    }
    const size_t sm_base = (size_t)2 * ((nwords + 1) & ~1) * sizeof(uint32_t);
    const bool use_smem = sm_base + (size_t)max_row * sizeof(int32_t) <= (size_t)96 * 1024;
    const size_t sm = use_smem ? sm_base + (size_t)max_row * sizeof(int32_t) : sm_base;
    DBuf<int64_t> cnt;
    DBuf<int32_t> cursor;
    cnt.alloc(std::max<int64_t>(L->ntiles, 1), s);
    L->s_ptr.alloc(L->ntiles + 1, s);
    if (!use_smem) cursor.alloc(std::max<int64_t>(L->ntiles, 1), s);
    GView gv{g.g_of.p, g.g_pos.p, g.g_ptr.p, g.g_mem.p, g.g_w.p};
    StackArgs sa{gv, L->cp.t_rp.p, L->cp.t_col.p, L->ap.t_rp.p, L->ap.t_col.p, bpat.t_rp.p, bpat.t_col.p,
                 sym_operands ? L->b_map.p : nullptr, cnt.p, nullptr, nullptr, nullptr, cursor.p, 0,
                 use_smem ? 1 : 0};
    allow_dyn_smem(k_gt_stack, sm);
    const unsigned grid = (unsigned)std::min<int64_t>(g.ngrp, (int64_t)num_sms() * 8);
    if (L->ntiles) {
        k_gt_stack<<<grid, 256, sm, s>>>(g.ngrp, sa, nwords);
        DBG_LAUNCH_CK();
    }
    scan_exclusive(cnt.p, L->s_ptr.p, L->ntiles, s);
    L->nentries = read_i64(L->s_ptr.p + L->ntiles, s);
    L->st_a.alloc(std::max<int64_t>(L->nentries, 1), s);
    L->st_b.alloc(std::max<int64_t>(L->nentries, 1), s);
    sa.fill = 1;
    sa.s_ptr = L->s_ptr.p;
    sa.st_a = L->st_a.p;
    sa.st_b = L->st_b.p;
    if (L->ntiles) {
        k_gt_stack<<<grid, 256, sm, s>>>(g.ngrp, sa, nwords);
        DBG_LAUNCH_CK();
    }
    L->a_pack.alloc(std::max<int64_t>(L->a_bytes, 16), s);
    if (!L->b_is_a) L->b_pack.alloc(std::max<int64_t>(L->b_bytes, 16), s);
    return L;
}

void lowtier_pack(LowTierPlan& L, dbcsr_matrix_* A, dbcsr_matrix_* B, cudaStream_t s) {
    const Groups& g = *L.groups;
    pack_operand(A, L.ap, L.a_off, L.a_bytes, L.a_pack, g, 0, L.nparts, s);
    if (!L.b_is_a) pack_operand(B, L.bp, L.b_off, L.b_bytes, L.b_pack, g, L.b_from_a_style ? 0 : 1, L.nparts, s);
}

void lowtier_run(LowTierPlan& L, dbcsr_matrix_* A, const LowTierOut& o, cudaStream_t s) {
    const Groups& g = *L.groups;
    if (!L.ntiles) return;
    LtArgs a{};
    a.ntiles = L.ntiles;
    a.c_trow = L.cp.t_row.p;
    a.c_tcol = L.cp.t_col.p;
    a.s_ptr = L.s_ptr.p;
    a.st_a = L.st_a.p;
    a.st_b = L.st_b.p;
    a.a_tkgrp = L.ap.t_col.p;
    a.a_pack = L.a_pack.p;
    a.a_off = L.a_off.p;
    a.b_pack = L.b_is_a ? L.a_pack.p : L.b_pack.p;
    a.b_off = L.b_is_a ? L.a_off.p : L.b_off.p;
    a.g = GView{g.g_of.p, g.g_pos.p, g.g_ptr.p, g.g_mem.p, g.g_w.p};
    a.bs = A->bs.p;
    a.f_rp = o.f_rp;
    a.f_col = o.f_col;
    a.f_comp = o.f_comp;
    a.f_off = o.f_off;
    a.f_cin = o.f_cin;
    a.ci_off = o.ci_off;
    a.ci_data = o.ci_data;
    a.alpha = o.alpha;
    a.beta = o.beta;
    a.c_data = o.c_data;
    a.c_norm = o.c_norm;
    a.c_dev2 = o.c_dev2;
    a.nparts = L.nparts;
    a.err = L.err.p;
    const size_t sm = sizeof(LtShared) + 1024;
    allow_dyn_smem(k_lowtier, sm);
    const unsigned grid = (unsigned)std::min<int64_t>(L.ntiles, (int64_t)num_sms());
    k_lowtier<<<grid, kLtThreads, sm, s>>>(a);
    DBG_LAUNCH_CK();
}

void lowtier_check(LowTierPlan& L, cudaStream_t s) {
    int e = 0;
    DBG_CK(cudaMemcpyAsync(&e, L.err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    DBG_CK(cudaStreamSynchronize(s));
    if (e == 1) fail(DBCSR_ETIMEOUT, "multiply: a wait of the tensor-core kernel ran out");
    if (e == 2) fail(DBCSR_EINVAL, "multiply: an operand declared symmetric has an asymmetric pattern");
}

int64_t lowtier_entries(const LowTierPlan& L) { return L.nentries; }
int64_t lowtier_tiles(const LowTierPlan& L) { return L.ntiles; }

}  // namespace dbg
