// Sharding a block matrix over several GPUs by block rows (the paper's DBCSR distributes
// block rows and columns over a 2-D process grid and multiplies with Cannon's algorithm and
// asynchronous point-to-point messages; section "DBCSR library").  Here a matrix is split
// into spatial domains of block rows, one per rank: a product C = A B needs, on each rank,
// the rows of B indexed by the block columns of its own rows of A -- its own rows plus a halo
// of neighbouring rows -- so one exchange of halo rows per product suffices, and scalars
// (residual, traces) take one sum over the ranks.
//
// Host-only functions (no GPU): the domain partition of the block rows and the halo lists.
// The partition needs no coordinates: recursive bisection of the block graph (blocks I, J
// adjacent when block (I, J) is present), each part ordered by breadth-first distance from a
// far block (a pseudo-peripheral vertex found by repeated sweeps) and cut at the weighted
// median, so that each domain is a compact region of the coupling graph.
#include <algorithm>
#include <climits>
#include <queue>
#include <string>
#include <vector>

#include "common.cuh"

namespace dbg {
namespace {

struct Graph {
    int32_t n;
    const int64_t* rp;
    const int32_t* col;
};

// Breadth-first distances from src inside the vertex set marked in `in` (others -1).
void bfs(const Graph& g, const std::vector<char>& in, int32_t src, std::vector<int32_t>& dist) {
    std::fill(dist.begin(), dist.end(), -1);
    std::queue<int32_t> q;
    dist[src] = 0;
    q.push(src);
    while (!q.empty()) {
        const int32_t v = q.front();
        q.pop();
        for (int64_t e = g.rp[v]; e < g.rp[v + 1]; ++e) {
            const int32_t w = g.col[e];
            if (in[w] && dist[w] < 0) {
                dist[w] = dist[v] + 1;
                q.push(w);
            }
        }
    }
}

// Splits `verts` into nparts domains, owners first .. first + nparts - 1.
void bisect(const Graph& g, std::vector<int32_t> verts, int32_t nparts, int32_t first, const std::vector<double>& w,
            std::vector<char>& in, std::vector<int32_t>& dist, int32_t* owner) {
    if (nparts <= 1 || verts.size() <= 1) {
        for (int32_t v : verts) owner[v] = first;
        return;
    }
    for (int32_t v : verts) in[v] = 1;
    // a far vertex: two sweeps from the smallest index (vertices of another component are
    // unreached and count as farthest)
    int32_t src = *std::min_element(verts.begin(), verts.end());
    for (int sweep = 0; sweep < 2; ++sweep) {
        bfs(g, in, src, dist);
        int32_t far = src;
        for (int32_t v : verts)
            if (dist[v] > dist[far] || (dist[v] == dist[far] && v < far)) far = v;
        src = far;
    }
    bfs(g, in, src, dist);
    for (int32_t v : verts) in[v] = 0;
    std::vector<int32_t> order = verts;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        const int32_t da = dist[a] < 0 ? INT32_MAX : dist[a], db = dist[b] < 0 ? INT32_MAX : dist[b];
        return da != db ? da < db : a < b;
    });
    const int32_t left = nparts / 2;
    double total = 0.0;
    for (int32_t v : order) total += w[v];
    const double target = total * (double)left / (double)nparts;
    double acc = 0.0;
    size_t cut = 0;
    while (cut < order.size() && acc + 0.5 * w[order[cut]] < target) acc += w[order[cut++]];
    cut = std::min(std::max<size_t>(cut, 1), order.size() - 1);
    std::vector<int32_t> a(order.begin(), order.begin() + cut), b(order.begin() + cut, order.end());
    bisect(g, std::move(a), left, first, w, in, dist, owner);
    bisect(g, std::move(b), nparts - left, first + left, w, in, dist, owner);
}

void check_pattern(int32_t nblk, const int64_t* rp, const int32_t* col) {
    if (nblk < 1 || !rp || !col) fail(DBCSR_EINVAL, "partition: need nblk >= 1, row pointers and columns");
    if (rp[0] != 0) fail(DBCSR_EINVAL, "partition: row pointers must start at 0");
    for (int32_t i = 0; i < nblk; ++i)
        if (rp[i + 1] < rp[i]) fail(DBCSR_EINVAL, "partition: row pointers decrease");
    for (int64_t e = 0; e < rp[nblk]; ++e)
        if (col[e] < 0 || col[e] >= nblk) fail(DBCSR_EINVAL, "partition: block column out of range");
}

template <class F>
dbcsr_status guard_host(F&& f) {
    try {
        f();
        set_last_error("");
        return DBCSR_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return DBCSR_ENOMEM;
    }
}

}  // namespace
}  // namespace dbg

extern "C" {

dbcsr_status dbcsr_partition_rows(int32_t nblk, const int64_t* row_ptr, const int32_t* col, int32_t nparts,
                                  int32_t* owner) {
    return dbg::guard_host([&] {
        dbg::check_pattern(nblk, row_ptr, col);
        if (nparts < 1 || nparts > nblk || !owner) dbg::fail(DBCSR_EINVAL, "partition: need 1 <= nparts <= nblk");
        // weight of a row: its blocks + 1 (the work of its products grows with them)
        std::vector<double> w(nblk);
        for (int32_t i = 0; i < nblk; ++i) w[i] = (double)(row_ptr[i + 1] - row_ptr[i]) + 1.0;
        std::vector<int32_t> all(nblk);
        for (int32_t i = 0; i < nblk; ++i) all[i] = i;
        std::vector<char> in(nblk, 0);
        std::vector<int32_t> dist(nblk, -1);
        dbg::bisect(dbg::Graph{nblk, row_ptr, col}, std::move(all), nparts, 0, w, in, dist, owner);
    });
}

dbcsr_status dbcsr_halo_rows(int32_t nblk, const int64_t* row_ptr, const int32_t* col, const int32_t* owner,
                             int32_t rank, int32_t* halo, int32_t cap, int32_t* n) {
    return dbg::guard_host([&] {
        dbg::check_pattern(nblk, row_ptr, col);
        if (!owner || !n || cap < 0 || (cap > 0 && !halo)) dbg::fail(DBCSR_EINVAL, "halo_rows: bad argument");
        std::vector<char> need(nblk, 0);
        for (int32_t i = 0; i < nblk; ++i) {
            if (owner[i] != rank) continue;
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
                if (owner[col[e]] != rank) need[col[e]] = 1;
        }
        int32_t k = 0;
        for (int32_t i = 0; i < nblk; ++i)
            if (need[i]) {
                if (k < cap) halo[k] = i;
                ++k;
            }
        *n = k;
    });
}

}  // extern "C"
