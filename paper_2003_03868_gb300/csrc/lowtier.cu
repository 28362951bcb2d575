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

#include "bf16split.cuh"
#include "common.cuh"
#include "tc05.cuh"

namespace dbg {

namespace {

constexpr int kTileRows = 128;                 // M of the MMA; rows of every packed tile
constexpr int kGroupRows = (kGroupWidth + 7) & ~7;          // packed rows of the widest group
constexpr int kRunMax = 2;                     // K steps per stage (one bulk copy per operand)
constexpr int kStageBytesMax = kRunMax * 2 * 2 * 2 * kGroupRows * 16;   // 28 KB
constexpr int kStages = 5;
constexpr int kOutStride = kTileRows - 15;     // 113 floats per staged output row (odd: no bank conflicts)
constexpr int kEpiWarps = 8;                   // two per TMEM lane quadrant
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kLoaderWarp = 2 + kEpiWarps;     // fetches the epilogue's tables one tile ahead
constexpr int kLtThreads = 64 + kEpiThreads + 32;   // producer, MMA, epilogue warps, table loader
constexpr int kAccs = 4;                       // TMEM accumulators of up to 128 columns
constexpr int kTmemCols = 128 * kAccs;
constexpr int kEpiBatch = 8;                   // C-input loads a lane issues before its first store
constexpr long long kWaitLimit = 4000000000ll; // about 2 s at 2 GHz

// ------------------------------------------------------------------ groups
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

// The kTop strongest off-diagonal couplings of every block row: one warp per row.  Every lane
// keeps the best kTop entries of its strided share (sorted by norm, descending, then column,
// ascending), then kTop rounds of a warp arg-max pop the row's best.  Slots the row cannot fill
// get a = -1.
constexpr int kTop = 12;
struct alignas(16) Coupling {
    double w;
    int32_t a, b;
};

__device__ __forceinline__ bool stronger(double w1, int32_t c1, double w2, int32_t c2) {
    return w1 > w2 || (w1 == w2 && c1 < c2);
}

__global__ void __launch_bounds__(256) k_top_couplings(int32_t nb, const int64_t* __restrict__ rp,
                                                       const int32_t* __restrict__ col,
                                                       const double* __restrict__ nrm, Coupling* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int32_t i = (int32_t)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    if (i >= nb) return;
    constexpr int32_t kNone = 0x7fffffff;
    double w[kTop];
    int32_t c[kTop];
#pragma unroll
    for (int k = 0; k < kTop; ++k) {
        w[k] = -1.0;                     // below every norm
        c[k] = kNone;
    }
    const int64_t q1 = rp[i + 1];
    for (int64_t q = rp[i] + lane; q < q1; q += 32) {
        int32_t nc = col[q];
        if (nc == i) continue;
        double nw = nrm[q];
        if (!stronger(nw, nc, w[kTop - 1], c[kTop - 1])) continue;
#pragma unroll
        for (int k = 0; k < kTop; ++k) {  // insertion: the displaced entry moves down
            if (stronger(nw, nc, w[k], c[k])) {
                const double tw = w[k];
                const int32_t tc = c[k];
                w[k] = nw;
                c[k] = nc;
                nw = tw;
                nc = tc;
            }
        }
    }
    Coupling* o = out + (size_t)i * kTop;
    int r = 0;
    for (; r < kTop; ++r) {
        double bw = w[0];
        int32_t bc = c[0];
#pragma unroll
        for (int sh = 16; sh; sh >>= 1) {
            const double ow = __shfl_xor_sync(0xffffffffu, bw, sh);
            const int32_t oc = __shfl_xor_sync(0xffffffffu, bc, sh);
            if (stronger(ow, oc, bw, bc)) {
                bw = ow;
                bc = oc;
            }
        }
        if (bc == kNone) break;          // the same on every lane
        if (lane == 0) o[r] = Coupling{bw, min(i, bc), max(i, bc)};
        if (c[0] == bc) {                // the one lane that held it (columns are unique in a row)
#pragma unroll
            for (int k = 0; k + 1 < kTop; ++k) {
                w[k] = w[k + 1];
                c[k] = c[k + 1];
            }
            w[kTop - 1] = -1.0;
            c[kTop - 1] = kNone;
        }
    }
    if (lane == 0)
        for (; r < kTop; ++r) o[r] = Coupling{0.0, -1, -1};
}

}  // namespace

std::shared_ptr<Groups> build_groups(dbcsr_matrix_* M) {
    check_finalized(M);
    ensure_norms(M);
    cudaStream_t s = M->stream;
    const int32_t nb = M->nblk;
    // candidate merges: the kTop strongest off-diagonal couplings of every block row, selected on
    // the device; only the selected couplings come to the host
    std::vector<Coupling> top((size_t)nb * kTop);
    if (nb > 0) {
        DBuf<Coupling> d_top;
        d_top.alloc((int64_t)nb * kTop, s);
        k_top_couplings<<<grid_for(nb, 8), 256, 0, s>>>(nb, M->rp.p, M->col.p, M->norms.p, d_top.p);
        DBG_LAUNCH_CK();
        DBG_CK(cudaMemcpyAsync(top.data(), d_top.p, sizeof(Coupling) * top.size(), cudaMemcpyDeviceToHost, s));
        DBG_CK(cudaStreamSynchronize(s));
    }
    std::vector<Coupling> edges;
    edges.reserve(top.size());
    for (const Coupling& e : top)
        if (e.a >= 0) edges.push_back(e);
    std::sort(edges.begin(), edges.end(), [](const Coupling& x, const Coupling& y) {
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
    for (const Coupling& e : edges) {
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
    std::vector<int32_t> fill(g_ptr.begin(), g_ptr.end() - 1), g_mrec(nb), g_midx(nb);
    int max_members = 0;
    for (int32_t i = 0; i < nb; ++i) {
        const int32_t k = g_of[i];
        g_midx[i] = fill[k] - g_ptr[k];
        g_mrec[fill[k]] = g_w[k] | (M->h_bs[i] << 8);
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
    g->g_mrec.alloc(nb, s);
    g->g_midx.alloc(nb, s);
    DBG_CK(cudaMemcpyAsync(g->g_mrec.p, g_mrec.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s));
    DBG_CK(cudaMemcpyAsync(g->g_midx.p, g_midx.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s));
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

__device__ __forceinline__ int lt_rows(int w) { return (w + 7) & ~7; }

// Packed bytes of every tile: ceil(width of its K group / 16) steps, each nparts x 2 chunks of
// (width of its row group, rounded up to 8) rows x 16 bytes.
__global__ void k_gt_bytes(int64_t nt, const int32_t* __restrict__ t_kgrp, const int32_t* __restrict__ t_rgrp,
                           const int32_t* __restrict__ g_w, int nparts, int64_t* __restrict__ bytes) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x)
        bytes[t] = (int64_t)lt_ksteps(g_w[t_kgrp[t]]) * nparts * 2 * lt_rows(g_w[t_rgrp[t]]) * 16;
}

// K steps of every tile that hold a nonzero column (bit s: columns 16 s .. 16 s + 15 of the
// tile's K group): a block (I, K) of an A-style tile covers K's columns; a transposed (B-role)
// tile's block (K, J) covers K's.  Steps with no block are all zero and are skipped.
__global__ void k_gt_kmask(int64_t nb, const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                           const int32_t* __restrict__ bs, const int32_t* __restrict__ g_pos,
                           const int32_t* __restrict__ blk_tile, int transpose, unsigned* __restrict__ kmask) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = blk_tile[b];
        if (t < 0) continue;
        const int32_t K = transpose ? row[b] : col[b];
        const int p0 = g_pos[K], p1 = p0 + bs[K] - 1;
        const unsigned bits = ((2u << (p1 >> 4)) - 1u) & ~((1u << (p0 >> 4)) - 1u);
        atomicOr(kmask + t, bits);
    }
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
struct PackArgs {
    int64_t nb;
    const int32_t* row; const int32_t* col; const int64_t* off; const double* data; const int32_t* bs;
    const int32_t* blk_tile; const int64_t* t_off;
    const int32_t* g_pos; const int32_t* g_of; const int32_t* g_w;
    int transpose;       // 0: block (I, K) -> rows of I, K columns of K; 1: block (K, J) -> rows of J, K of K
    int nparts;          // 1: plain BF16; 2: hi and lo
    uint8_t* pack;
};

// One warp per block: its elements into the tile, at (row, kcol) -> step kcol / 16, part (hi,
// lo), chunk (kcol / 8) % 2, row, element kcol % 8, with R = the tile's rows rounded up to 8:
// step s at s * nparts * 2 * R * 16 bytes, chunk at R * 16, row at 16.
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
        const int R = lt_rows(P.g_w[P.g_of[P.transpose ? J : I]]);
        const int slab = P.nparts * 2 * R * 16;
        // (i, j) of element e = i n + j, stepped by 32 elements without a division per element
        const int di = 32 / n, dj = 32 - di * n;
        int i = lane / n, j = lane - i * n;
        for (int e = lane; e < m * n; e += 32) {
            const int r = P.transpose ? pj + j : pi + i;
            const int kc = P.transpose ? pi + i : pj + j;
            const double x = src[e];
            uint8_t* p = base + (int64_t)(kc >> 4) * slab + ((kc >> 3) & 1) * (R * 16) + r * 16 + (kc & 7) * 2;
            if (P.nparts == 2) {
                uint16_t hi, lo;
                bf16_split(x, hi, lo);
                *(uint16_t*)p = hi;
                *(uint16_t*)(p + 2 * R * 16) = lo;
            } else {
                *(uint16_t*)p = bf16_bits(x);
            }
            i += di;
            j += dj;
            if (j >= n) {
                j -= n;
                ++i;
            }
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

// Per stack entry, what the kernel's producer and MMA warps need without dependent loads:
// ea = byte offset of the A tile | the K steps where both tiles hold a nonzero column (a bit
// mask; offsets are multiples of 4 KB), eb = byte offset of the B tile.
__global__ void k_lt_entry_meta(int64_t ne, const int32_t* __restrict__ st_a, const int32_t* __restrict__ st_b,
                                const unsigned* __restrict__ a_kmask, const unsigned* __restrict__ b_kmask,
                                const int64_t* __restrict__ a_off, const int64_t* __restrict__ b_off,
                                int64_t* __restrict__ ea, int64_t* __restrict__ eb) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t ta = st_a[e], tb = st_b[e];
        ea[e] = a_off[ta] | (int64_t)(a_kmask[ta] & b_kmask[tb] & 255u);
        eb[e] = b_off[tb];
    }
}

// The C tiles' tables: tbl[tile][member of I][member of J] = formed block k, for every formed
// block the product computes (the rest of the table holds -1).
__global__ void k_lt_ctable(int64_t nform, const int32_t* __restrict__ blk_tile, const int32_t* __restrict__ f_row,
                            const int32_t* __restrict__ f_col, const int32_t* __restrict__ g_midx,
                            int32_t* __restrict__ tbl) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nform; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = blk_tile[k];
        if (t < 0) continue;
        tbl[(int64_t)t * (kGroupMembers * kGroupMembers) + g_midx[f_row[k]] * kGroupMembers + g_midx[f_col[k]]] =
            (int32_t)k;
    }
}

// Work of the tensor-core kernel per C tile: live[t] = 1 if any K step of its stack is
// multiplied (a tile without one is written as zeros); and the sums over the executed K steps
// of 1, of N and of the copied rows, from which the MMA flops and the copied bytes follow.
__global__ void k_lt_work(int64_t ntiles, const int64_t* __restrict__ s_ptr, const int64_t* __restrict__ ea,
                          const int32_t* __restrict__ c_trow, const int32_t* __restrict__ c_tcol,
                          const int32_t* __restrict__ g_w, uint8_t* __restrict__ live,
                          unsigned long long* __restrict__ out) {
    unsigned long long ks = 0, ksn = 0, ksr = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
        const int wc = g_w[c_tcol[t]], wr = g_w[c_trow[t]];
        const int N = ((wc + 15) >> 4) << 4;
        const int rows = ((wr + 7) & ~7) + ((wc + 7) & ~7);
        unsigned long long k = 0;
        for (int64_t e = s_ptr[t]; e < s_ptr[t + 1]; ++e) k += (unsigned long long)__popcll(ea[e] & 255);
        live[t] = k ? 1 : 0;
        ks += k;
        ksn += k * N;
        ksr += k * rows;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ks += __shfl_xor_sync(0xffffffffu, ks, o);
        ksn += __shfl_xor_sync(0xffffffffu, ksn, o);
        ksr += __shfl_xor_sync(0xffffffffu, ksr, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (ks) atomicAdd(out, ks);
        if (ksn) atomicAdd(out + 1, ksn);
        if (ksr) atomicAdd(out + 2, ksr);
    }
}

// ------------------------------------------------------------------ the tensor-core kernel
struct LtArgs {
    int64_t ntiles;
    const int32_t* c_trow; const int32_t* c_tcol; const int64_t* s_ptr;
    const int64_t* ea; const int64_t* eb;    // per stack entry: A offset | K-step mask, B offset
    const uint8_t* t_live;                   // per C tile: 1 if any K step is multiplied
    const uint8_t* a_pack; const uint8_t* b_pack;
    GView g;
    const int32_t* g_mrec;                   // per member slot: first row | rows << 8
    const int32_t* c_tbl;                    // per C tile, 16 x 16: formed block of (row member, column member) or -1
    const int64_t* f_off; const int64_t* f_cin;
    const int64_t* ci_off; const double* ci_data;
    double alpha, beta;
    double* c_data; double* c_norm; double* c_dev2;
    int nparts;
    int* err;                                // 1: a wait ran out
};

// What the epilogue needs of one C tile: the atom blocks it writes and where.
struct LtTables {
    int64_t koff[kGroupMembers][kGroupMembers];   // element offset of the formed block
    int64_t kcin[kGroupMembers][kGroupMembers];   // element offset of its C input, -1 without
    int32_t tbl[kGroupMembers][kGroupMembers];    // formed block of (row member, column member) or -1
    int32_t rowblk[kGroupMembers], colblk[kGroupMembers];
    int32_t rowrec[kGroupMembers], colrec[kGroupMembers];   // first row | rows << 8
    int32_t nm, nn, wc, live;
};

struct LtShared {
    alignas(1024) uint8_t stage[kStages][kStageBytesMax];
    float out[kTileRows][kOutStride];        // the finished accumulator, staged for coalesced writes
    LtTables T[2];                           // filled by the loader warp, one tile ahead
    uint64_t full[kStages], empty[kStages], acc_full[kAccs], acc_empty[kAccs], fin;
    uint64_t tbl_full[2], tbl_empty[2];
    uint32_t tmem_base;
    int abort;                               // set once by a role whose wait ran out
    int epi_stop;                            // the epilogue's snapshot of abort
};

__device__ __forceinline__ void lt_epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }

__device__ __forceinline__ int lt_aborted(const LtShared& S) { return *(volatile const int*)&S.abort; }

__device__ __forceinline__ void lt_fail(const LtArgs& A, LtShared& S) {
    *(volatile int*)&S.abort = 1;
    atomicExch(A.err, 1);
}

// The next run of consecutive set bits of mask (at most kRunMax long): first bit and length.
__device__ __forceinline__ int lt_next_run(unsigned& mask, int& len) {
    const int k = __ffs(mask) - 1;
    len = 1;
    while (len < kRunMax && (mask & (1u << (k + len)))) ++len;
    mask &= ~(((1u << len) - 1u) << k);
    return k;
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
        for (int i = 0; i < kAccs; ++i) {
            tc::mbar_init(&S.acc_full[i], 1);
            tc::mbar_init(&S.acc_empty[i], kEpiThreads);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&S.tbl_full[i], 32);
            tc::mbar_init(&S.tbl_empty[i], 1);
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
    const int np = A.nparts;

    if (warp == 0) {
        // ---------------- producer: per stack entry, the K steps where both tiles are nonzero, in
        // runs of up to kRunMax consecutive steps, one bulk copy per operand and run.  A K step of
        // a tile with R rows (its group's width rounded up to 8) is np x 2 chunks of R x 16 bytes.
        // The warp fetches the metadata of 32 entries at once (one per lane); lane 0 issues.
        int stage = 0;
        uint32_t phase = 0;
        int64_t armed = 0;
        bool stop = false;
        for (int64_t t = blockIdx.x; t < A.ntiles && !stop; t += gridDim.x) {
            const int64_t e0 = A.s_ptr[t], e1 = A.s_ptr[t + 1];
            const int ra = lt_rows(A.g.g_w[A.c_trow[t]]), rb = lt_rows(A.g.g_w[A.c_tcol[t]]);
            const int sa_bytes = np * 2 * ra * 16, sb_bytes = np * 2 * rb * 16;
            for (int64_t eb0 = e0; eb0 < e1 && !stop; eb0 += 32) {
                const int64_t my = eb0 + lane;
                const int64_t mea = my < e1 ? A.ea[my] : 0, meb = my < e1 ? A.eb[my] : 0;
                const int cnt = (int)min((int64_t)32, e1 - eb0);
                for (int x = 0; x < cnt && !stop; ++x) {
                    const int64_t va = __shfl_sync(0xffffffffu, mea, x), vb = __shfl_sync(0xffffffffu, meb, x);
                    if (lane == 0) {
                        unsigned mask = (unsigned)(va & 255);
                        const uint8_t* pa = A.a_pack + (va & ~(int64_t)255);
                        const uint8_t* pb = A.b_pack + vb;
                        while (mask) {
                            int len;
                            const int k = lt_next_run(mask, len);
                            if (!tc::mbar_wait(&S.empty[stage], phase ^ 1u, kWaitLimit)) {
                                lt_fail(A, S);
                                break;
                            }
                            tc::mbar_arrive_expect_tx(&S.full[stage], (uint32_t)(len * (sa_bytes + sb_bytes)));
                            tc::bulk_g2s(S.stage[stage], pa + (int64_t)k * sa_bytes, (uint32_t)(len * sa_bytes),
                                         &S.full[stage]);
                            tc::bulk_g2s(S.stage[stage] + len * sa_bytes, pb + (int64_t)k * sb_bytes,
                                         (uint32_t)(len * sb_bytes), &S.full[stage]);
                            ++armed;
                            if (++stage == kStages) {
                                stage = 0;
                                phase ^= 1u;
                            }
                        }
                    }
                    stop = __shfl_sync(0xffffffffu, lt_aborted(S), 0) != 0;
                }
            }
        }
        // no copy may still be landing in shared memory when the CTA exits: wait (bounded)
        // for the last armed stages (after a normal run the MMA warp consumed them all)
        if (lane == 0)
            for (int64_t x = 0; x < armed && x < kStages; ++x) {
                if (--stage < 0) {
                    stage = kStages - 1;
                    phase ^= 1u;
                }
                if (!tc::mbar_wait(&S.full[stage], phase, kWaitLimit)) lt_fail(A, S);
            }
    } else if (warp == 1) {
        // ---------------- MMA issuer (lane 0): the same runs as the producer, np MMAs per K step
        // (hi*hi, then hi*lo and lo*hi for split operands); the warp fetches 32 entries' masks at once
        int stage = 0;
        uint32_t phase = 0;
        int it = 0;
        bool stop = false;
        for (int64_t t = blockIdx.x; t < A.ntiles && !stop; t += gridDim.x, ++it) {
            const int acc = it % kAccs;
            const uint32_t acc_phase = (uint32_t)(it / kAccs) & 1u;
            const int wc = A.g.g_w[A.c_tcol[t]];
            const int ra = lt_rows(A.g.g_w[A.c_trow[t]]), rb = lt_rows(wc);
            const int sa_bytes = np * 2 * ra * 16, sb_bytes = np * 2 * rb * 16;
            const uint32_t idesc = tc::instr_desc(1, kTileRows, ((wc + 15) >> 4) << 4);
            const uint32_t d_tmem = tmem + (uint32_t)(acc * 128);
            if (lane == 0) {
                if (!tc::mbar_wait(&S.acc_empty[acc], acc_phase ^ 1u, kWaitLimit)) lt_fail(A, S);
                tc::fence_after_sync();
            }
            stop = __shfl_sync(0xffffffffu, lt_aborted(S), 0) != 0;
            uint32_t accumulate = 0;
            const int64_t e0 = A.s_ptr[t], e1 = A.s_ptr[t + 1];
            for (int64_t eb0 = e0; eb0 < e1 && !stop; eb0 += 32) {
                const int64_t my = eb0 + lane;
                const unsigned mym = my < e1 ? (unsigned)(A.ea[my] & 255) : 0u;
                const int cnt = (int)min((int64_t)32, e1 - eb0);
                for (int x = 0; x < cnt && !stop; ++x) {
                    unsigned mask = __shfl_sync(0xffffffffu, mym, x);
                    if (lane == 0) {
                        while (mask) {
                            int len;
                            lt_next_run(mask, len);
                            if (!tc::mbar_wait(&S.full[stage], phase, kWaitLimit)) {
                                lt_fail(A, S);
                                break;
                            }
                            tc::fence_after_sync();
                            const uint32_t s0 = tc::smem_u32(S.stage[stage]);
                            for (int j = 0; j < len; ++j) {
                                const uint32_t sa = s0 + (uint32_t)(j * sa_bytes);
                                const uint32_t sb = s0 + (uint32_t)(len * sa_bytes + j * sb_bytes);
                                const uint64_t ah = tc::smem_desc(sa, ra * 16, 128);
                                const uint64_t bh = tc::smem_desc(sb, rb * 16, 128);
                                tc::mma_f16(d_tmem, ah, bh, idesc, accumulate);
                                accumulate = 1;
                                if (np == 2) {
                                    const uint64_t al = tc::smem_desc(sa + 2 * ra * 16, ra * 16, 128);
                                    const uint64_t bl = tc::smem_desc(sb + 2 * rb * 16, rb * 16, 128);
                                    tc::mma_f16(d_tmem, ah, bl, idesc, 1);
                                    tc::mma_f16(d_tmem, al, bh, idesc, 1);
                                }
                            }
                            tc::mma_commit(&S.empty[stage]);         // the stage is free once these MMAs ran
                            if (++stage == kStages) {
                                stage = 0;
                                phase ^= 1u;
                            }
                        }
                    }
                    stop = __shfl_sync(0xffffffffu, lt_aborted(S), 0) != 0;
                }
            }
            if (lane == 0) tc::mma_commit(&S.acc_full[acc]);      // the accumulator is complete
        }
        // every MMA this thread issued has completed before the TMEM is released
        if (lane == 0) {
            tc::mma_commit(&S.fin);
            if (!tc::mbar_wait(&S.fin, 0, kWaitLimit)) lt_fail(A, S);
        }
    } else if (warp == kLoaderWarp) {
        // ---------------- table loader: the tables of the epilogue's next tile, while it writes
        // the current one (every lane fetches 8 of the 256 member pairs, loads batched by level)
        constexpr int kPer = kGroupMembers * kGroupMembers / 32;
        int it = 0;
        for (int64_t t = blockIdx.x; t < A.ntiles; t += gridDim.x, ++it) {
            const int b = it & 1;
            const uint32_t ph = (uint32_t)(it >> 1) & 1u;
            int ok = 1;
            if (lane == 0) {
                ok = tc::mbar_wait(&S.tbl_empty[b], ph ^ 1u, kWaitLimit) ? 1 : 0;
                if (!ok) lt_fail(A, S);
            }
            if (!__shfl_sync(0xffffffffu, ok, 0) || __shfl_sync(0xffffffffu, lt_aborted(S), 0)) break;
            LtTables& T = S.T[b];
            const int32_t G = __ldg(A.c_trow + t), Gc = __ldg(A.c_tcol + t);
            int32_t k[kPer];
#pragma unroll
            for (int u = 0; u < kPer; ++u) k[u] = __ldg(A.c_tbl + t * (kGroupMembers * kGroupMembers) + 32 * u + lane);
            const int32_t m0 = __ldg(A.g.g_ptr + G), nm = __ldg(A.g.g_ptr + G + 1) - m0;
            const int32_t n0 = __ldg(A.g.g_ptr + Gc), nn = __ldg(A.g.g_ptr + Gc + 1) - n0;
            int64_t off[kPer], ci[kPer];
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                off[u] = k[u] >= 0 ? __ldg(A.f_off + k[u]) : 0;
                ci[u] = (k[u] >= 0 && A.f_cin) ? __ldg(A.f_cin + k[u]) : -1;
            }
            if (lane < nm) {
                T.rowblk[lane] = __ldg(A.g.g_mem + m0 + lane);
                T.rowrec[lane] = __ldg(A.g_mrec + m0 + lane);
            }
            if (lane < nn) {
                T.colblk[lane] = __ldg(A.g.g_mem + n0 + lane);
                T.colrec[lane] = __ldg(A.g_mrec + n0 + lane);
            }
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                const int p = 32 * u + lane;
                T.tbl[p >> 4][p & 15] = k[u];
                T.koff[p >> 4][p & 15] = off[u];
                T.kcin[p >> 4][p & 15] = ci[u] >= 0 ? __ldg(A.ci_off + ci[u]) : -1;
            }
            if (lane == 0) {
                T.nm = nm;
                T.nn = nn;
                T.wc = __ldg(A.g.g_w + Gc);
                T.live = __ldg(A.t_live + t);
            }
            tc::mbar_arrive(&S.tbl_full[b]);     // release: the stores above are visible to the waiters
        }
    } else {
        // ---------------- epilogue: warps 2..9.  The accumulator is staged in shared memory (a
        // warp reads TMEM lanes 32 * (warp % 4) .. and every other 16-column chunk), the TMEM
        // released, then each formed atom block is written by one warp, lanes over its contiguous
        // elements, with its norm summed in a fixed order.
        const int et = threadIdx.x - 64;                          // 0 .. kEpiThreads - 1
        const int q = warp & 3, ew = et >> 5, half = ew >> 2;
        const int r = 32 * q + lane;                              // tile row of this thread
        int it = 0;
        for (int64_t t = blockIdx.x; t < A.ntiles; t += gridDim.x, ++it) {
            if (et == 0) S.epi_stop = lt_aborted(S);
            lt_epi_sync();
            if (S.epi_stop) break;
            const int acc = it % kAccs;
            const uint32_t acc_phase = (uint32_t)(it / kAccs) & 1u;
            const int tb = it & 1;
            // the tile's tables (loader warp); a warp that did not see them complete skips the
            // tile's work but keeps to the barriers
            const bool tok = __all_sync(0xffffffffu, tc::mbar_wait(&S.tbl_full[tb], (uint32_t)(it >> 1) & 1u,
                                                                   kWaitLimit));
            if (!tok) lt_fail(A, S);
            const LtTables& T = S.T[tb];
            const int nm = tok ? T.nm : 0, nn = tok ? T.nn : 0;
            // every tile's accumulator phase completes (a tile without products commits no MMA
            // and is written as zeros, but its phase is still waited for); the TMEM loads are
            // warp-collective: a warp reads only if all its lanes saw the phase
            const bool empty = !tok || !T.live;
            const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&S.acc_full[acc], acc_phase, kWaitLimit)) && tok;
            if (!ok) lt_fail(A, S);
            tc::fence_after_sync();
            const int ncol = tok ? ((T.wc + 15) >> 4) << 4 : 0;
            for (int c0 = 16 * half; c0 < ncol; c0 += 32) {
                float v[16];
                if (!empty && ok) {
                    tc::tmem_ld16(tmem + (uint32_t)(acc * 128 + c0) + ((uint32_t)(32 * q) << 16), v);
                } else {
#pragma unroll
                    for (int x = 0; x < 16; ++x) v[x] = 0.f;
                }
#pragma unroll
                for (int x = 0; x < 16; ++x)
                    if (c0 + x < kOutStride) S.out[r][c0 + x] = v[x];
            }
            // the accumulator may be reused once every lane has read it
            tc::fence_before_sync();
            lt_epi_sync();
            tc::mbar_arrive(&S.acc_empty[acc]);
            if (ok) {
                for (int p = ew; p < nm * nn; p += kEpiWarps) {
                    const int a = p / nn, b = p - a * nn;
                    if (T.tbl[a][b] < 0) continue;
                    const int ra0 = T.rowrec[a] & 255, m = T.rowrec[a] >> 8;
                    const int cb0 = T.colrec[b] & 255, n = T.colrec[b] >> 8;
                    const bool diag = T.rowblk[a] == T.colblk[b];
                    double* __restrict__ out = A.c_data + T.koff[a][b];
                    const int64_t ci = T.kcin[a][b];
                    const double* __restrict__ cin = A.ci_data + (ci >= 0 ? ci : 0);
                    // (e + 1/2) / n is at least 1 / (2 n) away from an integer; the float
                    // product errs by far less for e < 2^14, so its truncation is e / n
                    const float rn = 1.0f / (float)n;
                    const int mn = m * n;
                    double sq = 0.0, d2 = 0.0;
                    for (int e0 = 0; e0 < mn; e0 += 32 * kEpiBatch) {
                        // the batch's C-input loads are all in flight before its first store
                        double c[kEpiBatch];
#pragma unroll
                        for (int u = 0; u < kEpiBatch; ++u) {
                            const int e = e0 + 32 * u + lane;
                            c[u] = (ci >= 0 && e < mn) ? __ldg(cin + e) : 0.0;
                        }
#pragma unroll
                        for (int u = 0; u < kEpiBatch; ++u) {
                            const int e = e0 + 32 * u + lane;
                            if (e < mn) {
                                const int i = (int)(((float)e + 0.5f) * rn), j = e - i * n;
                                double val = A.alpha * (double)S.out[ra0 + i][cb0 + j];
                                if (ci >= 0) val = val + A.beta * c[u];
                                out[e] = val;
                                sq = fma(val, val, sq);
                                // off the diagonal the distance to 1 is the norm (summed once
                                // below): the FP64 pipe, not the stores, would bound this loop
                                if (diag) {
                                    const double w = (i == j) ? val - 1.0 : val;
                                    d2 = fma(w, w, d2);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
                    if (diag) {
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) d2 += __shfl_xor_sync(0xffffffffu, d2, o);
                    } else {
                        d2 = sq;
                    }
                    if (lane == 0) {
                        const int32_t k = T.tbl[a][b];
                        A.c_norm[k] = sqrt(sq);
                        A.c_dev2[k] = d2;
                    }
                }
            }
            lt_epi_sync();
            if (et == 0) tc::mbar_arrive(&S.tbl_empty[tb]);      // the loader may refill these tables
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
int64_t tile_offsets(const TilePattern& P, const int32_t* t_kgrp, const int32_t* t_rgrp, const Groups& g, int nparts,
                     DBuf<int64_t>& off, cudaStream_t s) {
    DBuf<int64_t> bytes;
    bytes.alloc(std::max<int64_t>(P.nt, 1), s);
    off.alloc(P.nt + 1, s);
    if (P.nt) {
        k_gt_bytes<<<grid_for(P.nt, 256), 256, 0, s>>>(P.nt, t_kgrp, t_rgrp, g.g_w.p, nparts, bytes.p);
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
    int64_t ksteps = 0, ksteps_n = 0, ksteps_rows = 0;   // over the executed K steps: 1, N, copied rows
    DBuf<uint8_t> t_live;               // per C tile: 1 if any K step is multiplied
    DBuf<int64_t> ea, eb;               // per entry: A offset | K steps, B offset
    DBuf<int32_t> c_tbl;                // per C tile: 16 x 16 formed blocks
};

void lowtier_plan_delete(LowTierPlan* p) { delete p; }

namespace {

void pack_operand(const dbcsr_matrix_* M, const TilePattern& P, const DBuf<int64_t>& off, int64_t bytes,
                  DBuf<uint8_t>& pack, const Groups& g, int transpose, int nparts, cudaStream_t s) {
    if (!bytes || !M->nnzb) return;
    DBG_CK(cudaMemsetAsync(pack.p, 0, (size_t)bytes, s));
    PackArgs pa{M->nnzb, M->row.p, M->col.p, M->off.p, M->data.p, M->bs.p, P.blk_tile.p, off.p, g.g_pos.p,
                g.g_of.p, g.g_w.p, transpose, nparts, pack.p};
    k_gt_pack<<<grid_for(M->nnzb, 8), 256, 0, s>>>(pa);
    DBG_LAUNCH_CK();
}

}  // namespace

std::unique_ptr<LowTierPlan, void (*)(LowTierPlan*)> lowtier_prepare(int prec, dbcsr_matrix_* A, dbcsr_matrix_* B,
                                                                     std::shared_ptr<Groups> groups, bool sym_operands,
                                                                     int64_t nform, const int64_t* f_rp,
                                                                     const int32_t* f_row, const int32_t* f_col,
                                                                     const uint8_t* f_comp, cudaStream_t s) {
    std::unique_ptr<LowTierPlan, void (*)(LowTierPlan*)> L(new LowTierPlan(), lowtier_plan_delete);
    const Groups& g = *groups;
    L->groups = groups;
    L->nparts = prec == DBCSR_BF16X3 ? 2 : 1;
    if (g.ngrp > kMaxBlockRowsLt) fail(DBCSR_ECAPACITY, "multiply: too many groups for the tensor-core tier");
    // A: rows = A's group rows, K = its column groups
    L->ap = tile_pattern(g, A->rp.p, A->col.p, nullptr, A->nnzb, true, s);
    L->a_bytes = tile_offsets(L->ap, L->ap.t_col.p, L->ap.t_row.p, g, L->nparts, L->a_off, s);
    // B: symmetric operands read their K-major tiles from the A-style tiles of the transposed
    // position; otherwise B is packed transposed (rows = its column group, K = its row group)
    L->b_is_a = sym_operands && B == A;
    L->b_from_a_style = sym_operands;
    L->err.alloc(1, s);
    L->err.zero();
    if (!L->b_is_a) {
        L->bp = tile_pattern(g, B->rp.p, B->col.p, nullptr, B->nnzb, true, s);
        L->b_bytes = tile_offsets(L->bp, sym_operands ? L->bp.t_col.p : L->bp.t_row.p,
                                  sym_operands ? L->bp.t_row.p : L->bp.t_col.p, g, L->nparts, L->b_off, s);
    }
    const TilePattern& bpat = L->b_is_a ? L->ap : L->bp;
    if (sym_operands && bpat.nt) {
        L->b_map.alloc(bpat.nt, s);
        k_gt_transpose<<<grid_for(bpat.nt, 256), 256, 0, s>>>(bpat.nt, bpat.t_row.p, bpat.t_col.p, bpat.t_rp.p,
                                                               L->b_map.p, L->err.p);
        DBG_LAUNCH_CK();
    }
    // C tiles: group pairs of the atom blocks the product computes, and each tile's table of them
    L->cp = tile_pattern(g, f_rp, f_col, f_comp, nform, true, s);
    L->ntiles = L->cp.nt;
    L->c_tbl.alloc(std::max<int64_t>(L->ntiles, 1) * kGroupMembers * kGroupMembers, s);
    if (L->ntiles) {
        DBG_CK(cudaMemsetAsync(L->c_tbl.p, 0xff, sizeof(int32_t) * L->ntiles * kGroupMembers * kGroupMembers, s));
        k_lt_ctable<<<grid_for(nform, 256), 256, 0, s>>>(nform, L->cp.blk_tile.p, f_row, f_col, g.g_midx.p,
                                                          L->c_tbl.p);
        DBG_LAUNCH_CK();
    }
    L->cp.blk_tile.release();
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
    // nonzero K steps of every operand tile, and per entry those of both its tiles
    DBuf<unsigned> a_km, b_km;
    a_km.alloc(std::max<int64_t>(L->ap.nt, 1), s);
    a_km.zero();
    if (A->nnzb) {
        k_gt_kmask<<<grid_for(A->nnzb, 256), 256, 0, s>>>(A->nnzb, A->row.p, A->col.p, A->bs.p, g.g_pos.p,
                                                           L->ap.blk_tile.p, 0, a_km.p);
        DBG_LAUNCH_CK();
    }
    if (!L->b_is_a) {
        b_km.alloc(std::max<int64_t>(L->bp.nt, 1), s);
        b_km.zero();
        if (B->nnzb) {
            k_gt_kmask<<<grid_for(B->nnzb, 256), 256, 0, s>>>(B->nnzb, B->row.p, B->col.p, B->bs.p, g.g_pos.p,
                                                               L->bp.blk_tile.p, L->b_from_a_style ? 0 : 1, b_km.p);
            DBG_LAUNCH_CK();
        }
    }
    L->ea.alloc(std::max<int64_t>(L->nentries, 1), s);
    L->eb.alloc(std::max<int64_t>(L->nentries, 1), s);
    if (L->nentries) {
        k_lt_entry_meta<<<grid_for(L->nentries, 256), 256, 0, s>>>(
            L->nentries, L->st_a.p, L->st_b.p, a_km.p, L->b_is_a ? a_km.p : b_km.p, L->a_off.p,
            L->b_is_a ? L->a_off.p : L->b_off.p, L->ea.p, L->eb.p);
        DBG_LAUNCH_CK();
    }
    L->t_live.alloc(std::max<int64_t>(L->ntiles, 1), s);
    if (L->ntiles) {
        DBuf<int64_t> w;
        w.alloc(3, s);
        w.zero();
        k_lt_work<<<grid_for(L->ntiles, 256), 256, 0, s>>>(L->ntiles, L->s_ptr.p, L->ea.p, L->cp.t_row.p,
                                                            L->cp.t_col.p, g.g_w.p, L->t_live.p,
                                                            (unsigned long long*)w.p);
        DBG_LAUNCH_CK();
        int64_t h[3];
        DBG_CK(cudaMemcpyAsync(h, w.p, sizeof h, cudaMemcpyDeviceToHost, s));
        DBG_CK(cudaStreamSynchronize(s));
        L->ksteps = h[0];
        L->ksteps_n = h[1];
        L->ksteps_rows = h[2];
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
    a.ea = L.ea.p;
    a.eb = L.eb.p;
    a.t_live = L.t_live.p;
    a.a_pack = L.a_pack.p;
    a.b_pack = L.b_is_a ? L.a_pack.p : L.b_pack.p;
    a.g = GView{g.g_of.p, g.g_pos.p, g.g_ptr.p, g.g_mem.p, g.g_w.p};
    a.g_mrec = g.g_mrec.p;
    a.c_tbl = L.c_tbl.p;
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

int64_t lowtier_tiles(const LowTierPlan& L) { return L.ntiles; }
// split operands: three MMAs per K step (hi*hi, hi*lo, lo*hi); plain BF16: one
double lowtier_tensor_flops(const LowTierPlan& L) {
    return 2.0 * kTileRows * 16.0 * (double)L.ksteps_n * (L.nparts == 2 ? 3 : 1);
}
double lowtier_copy_bytes(const LowTierPlan& L) { return (double)L.ksteps_rows * L.nparts * 2 * 16; }

}  // namespace dbg
