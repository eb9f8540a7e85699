// Spatial-hash broad phase.
//
// Every triangle and edge is entered into a uniform grid (hashed cells) once
// per cell its box touches; entries are ordered by a stable radix sort on the
// bucket so the table is deterministic.  Each surface point (PT) and edge
// (EE) then visits the cells of its own box and tests the entries found
// there.  A pair found in several shared cells is emitted only from the cell
// that holds the minimum corner of the two boxes' intersection, so each pair
// appears exactly once without a dedup pass.  Primitives whose box spans more
// than kMaxCells cells are kept out of the grid ("oversize") and are tested by
// a direct loop instead.
#include "broadphase.cuh"

namespace zema {

constexpr double kMaxCells = 1024.0;       // entries spanning more cells stay out of the grid
constexpr double kMaxQueryCells = 32.0;    // queries spanning more cells run one block per query

struct Box6 {
    double lo[3], hi[3];
};

__device__ __forceinline__ long long cell_of(double v, double inv) { return (long long)floor(v * inv); }

__device__ __forceinline__ uint64_t pack_cell(long long cx, long long cy, long long cz) {
    const long long off = 1ll << 20;
    const uint64_t m = (1ull << 21) - 1;
    return ((uint64_t)(cx + off) & m) | (((uint64_t)(cy + off) & m) << 21) | (((uint64_t)(cz + off) & m) << 42);
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ Box6 ld_box(const double* b) {
    Box6 r;
    for (int k = 0; k < 3; ++k) {
        r.lo[k] = b[k];
        r.hi[k] = b[3 + k];
    }
    return r;
}

__device__ __forceinline__ bool overlap(const Box6& a, const Box6& b) {
    for (int k = 0; k < 3; ++k)
        if (a.lo[k] > b.hi[k] || b.lo[k] > a.hi[k]) return false;
    return true;
}

// box of n surface vertices (ids) over X0 (and X1), inflated by infl
__device__ __forceinline__ Box6 prim_box(const BPView& v, const int* ids, int n) {
    Box6 b;
    for (int k = 0; k < 3; ++k) {
        b.lo[k] = INFINITY;
        b.hi[k] = -INFINITY;
    }
    for (int i = 0; i < n; ++i) {
        const double* p = v.X0 + 3 * (size_t)ids[i];
        for (int k = 0; k < 3; ++k) {
            b.lo[k] = fmin(b.lo[k], p[k]);
            b.hi[k] = fmax(b.hi[k], p[k]);
        }
        if (v.X1) {
            const double* q = v.X1 + 3 * (size_t)ids[i];
            for (int k = 0; k < 3; ++k) {
                b.lo[k] = fmin(b.lo[k], q[k]);
                b.hi[k] = fmax(b.hi[k], q[k]);
            }
        }
    }
    for (int k = 0; k < 3; ++k) {
        b.lo[k] -= v.infl;
        b.hi[k] += v.infl;
    }
    return b;
}

__device__ __forceinline__ double box_cells(const Box6& b, double inv) {
    double n = 1.0;
    for (int k = 0; k < 3; ++k) n *= (double)(cell_of(b.hi[k], inv) - cell_of(b.lo[k], inv) + 1);
    return n;
}

// env of primitive i of kind 0 (surface vertex), 1 (edge), 2 (triangle)
__device__ __forceinline__ int prim_env(const BPView& v, int kind, int i) {
    const int sv = kind == 0 ? i : (kind == 1 ? v.edges[i].x : v.tris[i].x);
    return v.sv_env[sv];
}

__device__ __forceinline__ bool prim_skipped(const BPView& v, int kind, int i) {
    return v.env_skip && v.env_skip[prim_env(v, kind, i)];
}

// global id of local primitive 0 of a kind (0 points, 1 edges, 2 triangles)
__device__ __forceinline__ int base_of(const BPView& v, int kind) {
    return kind == 0 ? v.sv_base : (kind == 1 ? v.edge_base : v.tri_base);
}

// kind: 0 points, 1 edges, 2 tris.  For edges and tris also the grid entry
// count (0 when oversize) and the oversize flag.  Primitives of skipped envs
// get an empty box and no entries.
__global__ void k_boxes(BPView v, int kind, int n, double* box, int* cb, uint32_t* cnt, uint32_t* big) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int ids[3];
    int m;
    const int gi = i + base_of(v, kind);
    if (kind == 0) {
        ids[0] = gi;
        m = 1;
    } else if (kind == 1) {
        int2 e = v.edges[gi];
        ids[0] = e.x;
        ids[1] = e.y;
        m = 2;
    } else {
        int3 t = v.tris[gi];
        ids[0] = t.x;
        ids[1] = t.y;
        ids[2] = t.z;
        m = 3;
    }
    if (prim_skipped(v, kind, gi)) {
        for (int k = 0; k < 3; ++k) {
            box[6 * (size_t)i + k] = INFINITY;
            box[6 * (size_t)i + 3 + k] = -INFINITY;
            cb[6 * (size_t)i + k] = 1;
            cb[6 * (size_t)i + 3 + k] = 0;
        }
        if (cnt) {
            cnt[i] = 0u;
            big[i] = 0u;
        }
        return;
    }
    Box6 b = prim_box(v, ids, m);
    for (int k = 0; k < 3; ++k) {
        box[6 * (size_t)i + k] = b.lo[k];
        box[6 * (size_t)i + 3 + k] = b.hi[k];
        // integer cell range (the cell of a coordinate is monotone in it, so
        // the cell of max(lo_a, lo_b) is max(cell(lo_a), cell(lo_b)))
        cb[6 * (size_t)i + k] = (int)cell_of(b.lo[k], v.inv_cell);
        cb[6 * (size_t)i + 3 + k] = (int)cell_of(b.hi[k], v.inv_cell);
    }
    if (cnt) {
        double c = box_cells(b, v.inv_cell);
        bool o = !(c <= kMaxCells);  // non-finite boxes count as oversize too
        cnt[i] = o ? 0u : (uint32_t)c;
        big[i] = o ? 1u : 0u;
    }
}

// grid entries of one primitive family; bucket keys offset by bucket_base.
// kEmitLanes lanes per primitive, each taking every kEmitLanes-th cell of the
// box in x-fastest order (the entry order of the serial loop).
constexpr int kEmitLanes = 8;
__global__ void k_emit_entries(BPView v, int n, const int* cb, const uint32_t* off, uint32_t entry_base,
                               uint64_t bucket_base, uint64_t tmask, uint64_t* key, uint32_t* val,
                               uint64_t* cell_tmp, int* prim_tmp, int prim_flag) {
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(gt / kEmitLanes), l = (int)(gt % kEmitLanes);
    if (i >= n) return;
    const uint32_t o = off[i], e = off[i + 1];
    if (o == e) return;
    const int* c = cb + 6 * (size_t)i;
    const uint32_t nx = (uint32_t)(c[3] - c[0] + 1), ny = (uint32_t)(c[4] - c[1] + 1);
    for (uint32_t t = l; t < e - o; t += kEmitLanes) {
        const uint32_t txy = t % (nx * ny);
        const int cx = c[0] + (int)(txy % nx), cy = c[1] + (int)(txy / nx), cz = c[2] + (int)(t / (nx * ny));
        const uint32_t j = entry_base + o + t;
        uint64_t ck = pack_cell(cx, cy, cz);
        key[j] = bucket_base + (mix64(ck) & tmask);
        val[j] = j;
        cell_tmp[j] = ck;
        prim_tmp[j] = i | prim_flag;
    }
}

__global__ void k_gather_entries(const uint32_t* val, const uint64_t* cell_tmp, const int* prim_tmp, uint64_t* ecell,
                                 int* eprim, uint32_t n) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t s = val[j];
    ecell[j] = cell_tmp[s];
    eprim[j] = prim_tmp[s];
}

__global__ void k_bucket_ranges(const uint64_t* key, uint32_t n, uint32_t* bstart, uint32_t* bend) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint64_t b = key[j];
    if (j == 0 || key[j - 1] != b) bstart[b] = j;
    if (j == n - 1 || key[j + 1] != b) bend[b] = j + 1;
}

__global__ void k_compact_flags(const uint32_t* flag, const uint32_t* off, uint32_t sub, int n, int* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (flag[i]) out[off[i] - sub] = i;
}

__device__ __forceinline__ bool pair_ok(const BPView& v, int sa, int sb) {
    if (v.sv_env[sa] != v.sv_env[sb]) return false;
    int ba = v.sv_body[sa], bb = v.sv_body[sb];
    int ca = v.body_class[ba], cb = v.body_class[bb];
    if (ca >= 2 && cb >= 2) return false;
    if (ba == bb && ca != 0) return false;
    return true;
}

__device__ __forceinline__ bool pt_ok(const BPView& v, int p, int t) {
    int3 T = v.tris[t];
    if (p == T.x || p == T.y || p == T.z) return false;
    return pair_ok(v, p, T.x);
}

__device__ __forceinline__ bool ee_ok(const BPView& v, int a, int b) {
    int2 A = v.edges[a], B = v.edges[b];
    if (A.x == B.x || A.x == B.y || A.y == B.x || A.y == B.y) return false;
    return pair_ok(v, A.x, B.x);
}

// env of a query (kind 0: point, 1: edge)
__device__ __forceinline__ int query_env(const BPView& v, int kind, int q) {
    return v.sv_env[kind == 0 ? q : v.edges[q].x];
}

// local entry range [lo, hi) of the env of (global) query q (kind 0 queries
// meet triangles, kind 1 edges); the whole table when the primitives are not
// ordered by env
__device__ __forceinline__ void env_entries(const BPView& v, int kind, int q, int n_all, int& lo, int& hi) {
    const int* st = kind == 0 ? v.env_tri_start : v.env_edge_start;
    if (!st) {
        lo = 0;
        hi = n_all;
        return;
    }
    const int e = query_env(v, kind, q), eb = kind == 0 ? v.tri_base : v.edge_base;
    lo = st[e] - eb;
    hi = st[e + 1] - eb;
}

// first index k of the ascending list a[0..n) with a[k] >= x
__device__ __forceinline__ int lower_bound_i(const int* a, int n, int x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (a[m] < x)
            lo = m + 1;
        else
            hi = m;
    }
    return lo;
}

struct Table {
    const uint64_t* ecell;
    const int* eprim;
    const uint32_t* bstart;
    const uint32_t* bend;
    uint64_t bucket_base, tmask;
};

// kind 0: point queries against the triangle table; kind 1: edge queries
// against the edge table (only pairs with query < entry).  kQueryLanes lanes
// per query stride over each cell's bucket; a ballot places the group's hits
// in entry order, so the output is the serial visiting order (cells in
// z, y, x order, entries in table order, then the oversize list).
//
// WRITE false: the counting pass.  It also keeps the first kQuerySlots hits
// of each query, in order, in the query's slots (slots[kQuerySlots q ..]);
// k_slots_out then moves the queries whose hits all fit into the output, and
// the WRITE pass walks again only the queries with more hits (cnt[q] >
// kQuerySlots), so most queries are walked once.
constexpr int kQueryLanes = 8;  // a power of two below 32 (most buckets hold a few entries)
static_assert(kQueryLanes < 32 && (kQueryLanes & (kQueryLanes - 1)) == 0, "query group: power of two below 32");
constexpr int kQuerySlots = 8;
template <bool WRITE>
__global__ void k_query(BPView v, int kind, int nq, const double* qbox, const double* ebox_all, const int* qcb,
                        const int* ecb_all, Table T, const int* big, int nbig, int n_entries_all, uint32_t* cnt,
                        const uint32_t* off, int2* out) {
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = (int)(gt / kQueryLanes), l = (int)(gt % kQueryLanes);
    if (q >= nq) return;  // the whole group
    // global ids of the query and of local entry 0
    const int qg = q + base_of(v, kind), eb = kind == 0 ? v.tri_base : v.edge_base;
    if (prim_skipped(v, kind, qg)) {
        if (!WRITE && l == 0) cnt[q] = 0;
        return;
    }
    if (WRITE && cnt[q] <= (uint32_t)kQuerySlots) return;  // already out of its slots (or a large query)
    constexpr unsigned kGroupBits = (1u << kQueryLanes) - 1u;
    const unsigned gshift = threadIdx.x & (32u - kQueryLanes);
    const unsigned gmask = kGroupBits << gshift;
    Box6 a = ld_box(qbox + 6 * (size_t)q);
    double nc = box_cells(a, v.inv_cell);
    if (!(nc <= kMaxQueryCells)) {
        // large query: handled by k_query_big (one block per query)
        if (!WRITE && l == 0) cnt[q] = 0;
        return;
    }
    uint32_t c = 0;  // hits so far, the same in all lanes of the group
    const uint32_t o = WRITE ? off[q] : (uint32_t)kQuerySlots * (uint32_t)q;
    auto emit = [&](bool hit, int e) {
        const unsigned b = (__ballot_sync(gmask, hit) >> gshift) & kGroupBits;
        const uint32_t at = c + __popc(b & ((1u << l) - 1u));
        if (hit && (WRITE || at < (uint32_t)kQuerySlots)) out[o + at] = make_int2(qg, e + eb);
        c += __popc(b);
    };
    auto test = [&](int e) -> bool {
        if (kind == 0) return pt_ok(v, qg, e + eb);
        return q < e && ee_ok(v, qg, e + eb);
    };
    int qc[6];
    for (int k = 0; k < 6; ++k) qc[k] = qcb[6 * (size_t)q + k];
    for (int cz = qc[2]; cz <= qc[5]; ++cz)
        for (int cy = qc[1]; cy <= qc[4]; ++cy)
            for (int cx = qc[0]; cx <= qc[3]; ++cx) {
                uint64_t ck = pack_cell(cx, cy, cz);
                uint64_t bkt = T.bucket_base + (mix64(ck) & T.tmask);
                const uint32_t s = T.bstart[bkt], f = T.bend[bkt];
                for (uint32_t j0 = s; j0 < f; j0 += kQueryLanes) {
                    const uint32_t j = j0 + l;
                    bool hit = false;
                    int e = 0;
                    if (j < f && T.ecell[j] == ck) {
                        e = T.eprim[j];
                        // emit only from the cell holding the min corner of the
                        // boxes' intersection (integer test)
                        const int* ec = ecb_all + 6 * (size_t)e;
                        if (!(kind == 1 && e <= q) && max(qc[0], ec[0]) == cx && max(qc[1], ec[1]) == cy &&
                            max(qc[2], ec[2]) == cz) {
                            Box6 b = ld_box(ebox_all + 6 * (size_t)e);
                            hit = overlap(a, b) && test(e);
                        }
                    }
                    emit(hit, e);
                }
            }
    // the oversize entries (ascending ids) of the query's env
    int b_lo = 0, b_hi = nbig;
    if (v.env_tri_start) {
        int lo, hi;
        env_entries(v, kind, qg, n_entries_all, lo, hi);
        b_lo = lower_bound_i(big, nbig, lo);
        b_hi = lower_bound_i(big, nbig, hi);
    }
    for (int k0 = b_lo; k0 < b_hi; k0 += kQueryLanes) {
        const int k = k0 + l;
        bool hit = false;
        int e = 0;
        if (k < b_hi) {
            e = big[k];
            if (!(kind == 1 && e <= q)) {
                Box6 b = ld_box(ebox_all + 6 * (size_t)e);
                hit = overlap(a, b) && test(e);
            }
        }
        emit(hit, e);
    }
    if (!WRITE && l == 0) cnt[q] = c;
}

// Queries whose hits all fit their slots: the hits into the output at the
// query's offset, in order (large queries, flagged in big_flag, are left to
// k_query_big; queries with more hits to the WRITE pass of k_query).
__global__ void k_slots_out(int nq, const uint32_t* cnt, const uint32_t* off, const uint32_t* big_flag,
                            const int2* slots, int2* out) {
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = (int)(gt / kQuerySlots), j = (int)(gt % kQuerySlots);
    if (q >= nq || big_flag[q]) return;
    const uint32_t c = cnt[q];
    if (c > (uint32_t)kQuerySlots || (uint32_t)j >= c) return;
    out[off[q] + j] = slots[(size_t)kQuerySlots * q + j];
}

// Block-wide placement: each thread counts the hits of its items, an
// exclusive scan in thread order gives each thread its first output slot, and
// a second pass writes (so the output is in item order).  Returns the total.
template <bool WRITE, class Count, class Write>
__device__ __forceinline__ uint32_t block_place(uint32_t* sc, uint32_t base, Count count, Write write) {
    const uint32_t c = count();
    sc[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const uint32_t x = sc[t];
            sc[t] = run;
            run += x;
        }
        sc[blockDim.x] = run;
    }
    __syncthreads();
    if (WRITE) write(base + sc[threadIdx.x]);
    const uint32_t total = sc[blockDim.x];
    __syncthreads();
    return total;
}

// Oversize queries (boxes over kMaxQueryCells cells): one block per query.
//  - Up to kWalkCells cells, and at most a quarter as many cells as the env
//    has entries: the block walks the query's cells (thread t a
//    contiguous run of them in z, y, x order) through the grid exactly as
//    k_query does, then the oversize-entry list of the query's env; hits in
//    cell order, then list order.
//  - Otherwise: thread t tests the contiguous entry range [lo + t c,
//    lo + (t + 1) c) of the query's env (the whole table without env ranges);
//    hits in entry order.
constexpr double kWalkCells = 8192.0;
template <bool WRITE>
__global__ void k_query_big(BPView v, int kind, const int* qlist, const double* qbox, const double* ebox_all,
                            int n_entries_all, uint32_t* cnt, const uint32_t* off, int2* out, const int* qcb,
                            const int* ecb_all, Table T, const int* big, int nbig) {
    __shared__ uint32_t sc[257];
    const int q = qlist[blockIdx.x];
    // global ids of the query and of local entry 0
    const int qg = q + base_of(v, kind), eb = kind == 0 ? v.tri_base : v.edge_base;
    const Box6 a = ld_box(qbox + 6 * (size_t)q);
    const uint32_t base = WRITE ? off[q] : 0u;
    auto test = [&](int e) -> bool {
        if (kind == 1 && e <= q) return false;
        Box6 b = ld_box(ebox_all + 6 * (size_t)e);
        if (!overlap(a, b)) return false;
        return kind == 0 ? pt_ok(v, qg, e + eb) : ee_ok(v, qg, e + eb);
    };
    const double ncell = box_cells(a, v.inv_cell);
    int lo, hi;
    env_entries(v, kind, qg, n_entries_all, lo, hi);  // other envs' entries never pair
    // walk the cells only where that is clearly less work than the scan
    if (ncell <= kWalkCells && 4.0 * ncell <= (double)(hi - lo)) {
        int qc[6];
        for (int k = 0; k < 6; ++k) qc[k] = qcb[6 * (size_t)q + k];
        const int nx = qc[3] - qc[0] + 1, ny = qc[4] - qc[1] + 1, nz = qc[5] - qc[2] + 1;
        const int nc = nx * ny * nz;
        const int chunk = (nc + (int)blockDim.x - 1) / (int)blockDim.x;
        const int c0 = threadIdx.x * chunk, c1 = min(c0 + chunk, nc);
        // hits of one grid cell (linear index li), emitted through f
        auto cell_hits = [&](int li, auto f) {
            const int cx = qc[0] + li % nx, cy = qc[1] + (li / nx) % ny, cz = qc[2] + li / (nx * ny);
            const uint64_t ck = pack_cell(cx, cy, cz);
            const uint64_t bkt = T.bucket_base + (mix64(ck) & T.tmask);
            const uint32_t s0 = T.bstart[bkt], s1 = T.bend[bkt];
            for (uint32_t j = s0; j < s1; ++j) {
                if (T.ecell[j] != ck) continue;
                const int e = T.eprim[j];
                if (kind == 1 && e <= q) continue;
                const int* ec = ecb_all + 6 * (size_t)e;
                // emit only from the cell holding the min corner of the boxes' intersection
                if (max(qc[0], ec[0]) != cx || max(qc[1], ec[1]) != cy || max(qc[2], ec[2]) != cz) continue;
                if (test(e)) f(e);
            }
        };
        const uint32_t n_grid = block_place<WRITE>(
            sc, base,
            [&]() {
                uint32_t c = 0;
                for (int li = c0; li < c1; ++li) cell_hits(li, [&](int) { ++c; });
                return c;
            },
            [&](uint32_t o) {
                for (int li = c0; li < c1; ++li) cell_hits(li, [&](int e) { out[o++] = make_int2(qg, e + eb); });
            });
        // oversize entries (not in the grid), ascending ids, the query's env
        int b_lo = 0, b_hi = nbig;
        if (v.env_tri_start) {
            b_lo = lower_bound_i(big, nbig, lo);
            b_hi = lower_bound_i(big, nbig, hi);
        }
        const int bchunk = (b_hi - b_lo + (int)blockDim.x - 1) / (int)blockDim.x;
        const int k0 = b_lo + threadIdx.x * bchunk, k1 = min(k0 + bchunk, b_hi);
        const uint32_t n_big = block_place<WRITE>(
            sc, base + n_grid,
            [&]() {
                uint32_t c = 0;
                for (int k = k0; k < k1; ++k) c += test(big[k]) ? 1u : 0u;
                return c;
            },
            [&](uint32_t o) {
                for (int k = k0; k < k1; ++k)
                    if (test(big[k])) out[o++] = make_int2(qg, big[k] + eb);
            });
        if (!WRITE && threadIdx.x == 0) cnt[q] = n_grid + n_big;
        return;
    }
    const int chunk = (hi - lo + (int)blockDim.x - 1) / (int)blockDim.x;
    const int e0 = lo + threadIdx.x * chunk, e1 = min(e0 + chunk, hi);
    const uint32_t n = block_place<WRITE>(
        sc, base,
        [&]() {
            uint32_t c = 0;
            for (int e = e0; e < e1; ++e) c += test(e) ? 1u : 0u;
            return c;
        },
        [&](uint32_t o) {
            for (int e = e0; e < e1; ++e)
                if (test(e)) out[o++] = make_int2(qg, e + eb);
        });
    if (!WRITE && threadIdx.x == 0) cnt[q] = n;
}

// large-query flag of point or edge query boxes (never for skipped envs)
__global__ void k_query_flag(BPView v, int kind, const double* box, int n, uint32_t* flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (prim_skipped(v, kind, i + base_of(v, kind))) {
        flag[i] = 0u;
        return;
    }
    Box6 a = ld_box(box + 6 * (size_t)i);
    flag[i] = box_cells(a, v.inv_cell) <= kMaxQueryCells ? 0u : 1u;
}

static uint64_t pow2_at_least(uint64_t n) {
    uint64_t p = 64;
    while (p < n) p <<= 1;
    return p;
}

BroadPhase::~BroadPhase() {
    if (h_counts) cudaFreeHost(h_counts);
}

void BroadPhase::run(Allocator* A, const BPView& v, cudaStream_t st) {
    if (!h_counts) ZCHECK(cudaMallocHost(&h_counts, 16 * sizeof(uint32_t)));
    const int TB = 128;
    int nsv = v.nsv, ne = v.ne, nt = v.nt;
    pbox.ensure(A, 6 * (size_t)nsv + 6);
    ebox.ensure(A, 6 * (size_t)ne + 6);
    tbox.ensure(A, 6 * (size_t)nt + 6);
    tcnt.ensure(A, nt + 1);
    toff.ensure(A, nt + 2);
    ecnt.ensure(A, ne + 1);
    eoff.ensure(A, ne + 2);
    flag.ensure(A, (size_t)nt + ne + 2);
    flagoff.ensure(A, (size_t)nt + ne + 4);
    size_t mx = (size_t)nt + 2 * (size_t)ne + nsv + 16;
    tmp.ensure(A, scan_tmp_size(mx));
    pcb.ensure(A, 6 * (size_t)nsv + 6);
    ecb.ensure(A, 6 * (size_t)ne + 6);
    tcb.ensure(A, 6 * (size_t)nt + 6);
    if (nsv) ZL(k_boxes, div_up(nsv, TB), TB, 0, st)(v, 0, nsv, pbox.p, pcb.p, nullptr, nullptr);
    if (ne) ZL(k_boxes, div_up(ne, TB), TB, 0, st)(v, 1, ne, ebox.p, ecb.p, ecnt.p, flag.p + nt);
    if (nt) ZL(k_boxes, div_up(nt, TB), TB, 0, st)(v, 2, nt, tbox.p, tcb.p, tcnt.p, flag.p);
    ZLAUNCH();
    exclusive_scan(tcnt.p, toff.p, nt, tmp.p, st);
    exclusive_scan(ecnt.p, eoff.p, ne, tmp.p, st);
    // oversize lists: flags of tris [0, nt) and edges [nt, nt + ne)
    exclusive_scan(flag.p, flagoff.p, (size_t)nt + ne, tmp.p, st);
    ZCHECK(cudaMemcpyAsync(h_counts + 0, toff.p + nt, 4, cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaMemcpyAsync(h_counts + 1, eoff.p + ne, 4, cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaMemcpyAsync(h_counts + 2, flagoff.p + nt, 4, cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaMemcpyAsync(h_counts + 3, flagoff.p + nt + ne, 4, cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaStreamSynchronize(st));
    uint32_t Et = h_counts[0], Ee = h_counts[1], nbt = h_counts[2], nbe = h_counts[3] - h_counts[2];
    big_t.ensure(A, nbt + 1);
    big_e.ensure(A, nbe + 1);
    if (nt) ZL(k_compact_flags, div_up(nt, TB), TB, 0, st)(flag.p, flagoff.p, 0u, nt, big_t.p);
    // edge flag offsets continue after the triangles': subtract their count
    if (ne) ZL(k_compact_flags, div_up(ne, TB), TB, 0, st)(flag.p + nt, flagoff.p + nt, nbt, ne, big_e.p);
    ZLAUNCH();
    // grid tables: triangle buckets [0, Tt), edge buckets [Tt, Tt + Te)
    uint64_t Tt = pow2_at_least(2ull * Et + 1), Te = pow2_at_least(2ull * Ee + 1);
    size_t E = (size_t)Et + Ee;
    key.ensure(A, E + 1);
    key2.ensure(A, E + 1);
    val.ensure(A, E + 1);
    val2.ensure(A, E + 1);
    // the second key/val buffers double as the unsorted cell / prim scratch
    DBuf<uint64_t>& cell_tmp = ecell;
    cell_tmp.ensure(A, 2 * E + 2);
    eprim.ensure(A, 2 * E + 2);
    uint64_t* ctmp = cell_tmp.p + E + 1;
    int* ptmp = eprim.p + E + 1;
    bstart.ensure(A, Tt + Te);
    bend.ensure(A, Tt + Te);
    ZCHECK(cudaMemsetAsync(bstart.p, 0, (Tt + Te) * sizeof(uint32_t), st));
    ZCHECK(cudaMemsetAsync(bend.p, 0, (Tt + Te) * sizeof(uint32_t), st));
    if (nt) ZL(k_emit_entries, div_up((size_t)nt * kEmitLanes, TB), TB, 0, st)(v, nt, tcb.p, toff.p, 0, 0, Tt - 1, key.p, val.p, ctmp, ptmp, 0);
    if (ne) ZL(k_emit_entries, div_up((size_t)ne * kEmitLanes, TB), TB, 0, st)(v, ne, ecb.p, eoff.p, Et, Tt, Te - 1, key.p, val.p, ctmp, ptmp, 0);
    ZLAUNCH();
    if (E) {
        int bits = 1;
        while ((1ull << bits) < Tt + Te) ++bits;
        tmp.ensure(A, std::max(scan_tmp_size(mx), radix_tmp_size(E)));
        radix_sort(key.p, val.p, key2.p, val2.p, E, bits, tmp.p, st);
        ZL(k_gather_entries, div_up(E, 256), 256, 0, st)(val.p, ctmp, ptmp, cell_tmp.p, eprim.p, (uint32_t)E);
        ZL(k_bucket_ranges, div_up(E, 256), 256, 0, st)(key.p, (uint32_t)E, bstart.p, bend.p);
        ZLAUNCH();
    }
    Table TT{cell_tmp.p, eprim.p, bstart.p, bend.p, 0, Tt - 1};
    Table TE{cell_tmp.p, eprim.p, bstart.p, bend.p, Tt, Te - 1};
    qcnt_pt.ensure(A, nsv + 1);
    qoff_pt.ensure(A, nsv + 2);
    qcnt_ee.ensure(A, ne + 1);
    qoff_ee.ensure(A, ne + 2);
    // large queries (boxes over kMaxQueryCells cells): points, then edges
    pflag.ensure(A, (size_t)nsv + ne + 1);
    pflagoff.ensure(A, (size_t)nsv + ne + 2);
    if (nsv) ZL(k_query_flag, div_up(nsv, TB), TB, 0, st)(v, 0, pbox.p, nsv, pflag.p);
    if (ne) ZL(k_query_flag, div_up(ne, TB), TB, 0, st)(v, 1, ebox.p, ne, pflag.p + nsv);
    ZLAUNCH();
    exclusive_scan(pflag.p, pflagoff.p, (size_t)nsv + ne, tmp.p, st);
    ZCHECK(cudaMemcpyAsync(h_counts + 6, pflagoff.p + nsv, 4, cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaMemcpyAsync(h_counts + 7, pflagoff.p + nsv + ne, 4, cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaStreamSynchronize(st));
    uint32_t nbp = h_counts[6], nbq = h_counts[7] - h_counts[6];
    big_p.ensure(A, nbp + 1);
    big_q.ensure(A, nbq + 1);
    if (nsv) ZL(k_compact_flags, div_up(nsv, TB), TB, 0, st)(pflag.p, pflagoff.p, 0u, nsv, big_p.p);
    if (ne) ZL(k_compact_flags, div_up(ne, TB), TB, 0, st)(pflag.p + nsv, pflagoff.p + nsv, nbp, ne, big_q.p);
    ZLAUNCH();
    slot_pt.ensure(A, (size_t)kQuerySlots * nsv + 1);
    slot_ee.ensure(A, (size_t)kQuerySlots * ne + 1);
    if (nsv)
        ZL(k_query<false>, div_up((size_t)nsv * kQueryLanes, TB), TB, 0, st)(v, 0, nsv, pbox.p, tbox.p, pcb.p, tcb.p, TT, big_t.p, (int)nbt, nt,
                                                       qcnt_pt.p, nullptr, slot_pt.p);
    if (ne)
        ZL(k_query<false>, div_up((size_t)ne * kQueryLanes, TB), TB, 0, st)(v, 1, ne, ebox.p, ebox.p, ecb.p, ecb.p, TE, big_e.p, (int)nbe, ne,
                                                      qcnt_ee.p, nullptr, slot_ee.p);
    if (nbp)
        ZL(k_query_big<false>, nbp, 256, 0, st)(v, 0, big_p.p, pbox.p, tbox.p, nt, qcnt_pt.p, nullptr, nullptr, pcb.p,
                                                tcb.p, TT, big_t.p, (int)nbt);
    if (nbq)
        ZL(k_query_big<false>, nbq, 256, 0, st)(v, 1, big_q.p, ebox.p, ebox.p, ne, qcnt_ee.p, nullptr, nullptr, ecb.p,
                                                ecb.p, TE, big_e.p, (int)nbe);
    ZLAUNCH();
    tmp.ensure(A, std::max(scan_tmp_size(mx), E ? radix_tmp_size(E) : 0));
    exclusive_scan(qcnt_pt.p, qoff_pt.p, nsv, tmp.p, st);
    exclusive_scan(qcnt_ee.p, qoff_ee.p, ne, tmp.p, st);
    ZCHECK(cudaMemcpyAsync(h_counts + 4, qoff_pt.p + nsv, 4, cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaMemcpyAsync(h_counts + 5, qoff_ee.p + ne, 4, cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaStreamSynchronize(st));
    n_pt = h_counts[4];
    n_ee = h_counts[5];
    pt.ensure(A, n_pt + 1);
    ee.ensure(A, n_ee + 1);
    if (nsv && n_pt) {
        ZL(k_slots_out, div_up((size_t)nsv * kQuerySlots, TB), TB, 0, st)(nsv, qcnt_pt.p, qoff_pt.p, pflag.p, slot_pt.p,
                                                                         pt.p);
        ZL(k_query<true>, div_up((size_t)nsv * kQueryLanes, TB), TB, 0, st)(v, 0, nsv, pbox.p, tbox.p, pcb.p, tcb.p, TT, big_t.p, (int)nbt, nt,
                                                      qcnt_pt.p, qoff_pt.p, pt.p);
    }
    if (ne && n_ee) {
        ZL(k_slots_out, div_up((size_t)ne * kQuerySlots, TB), TB, 0, st)(ne, qcnt_ee.p, qoff_ee.p, pflag.p + nsv,
                                                                        slot_ee.p, ee.p);
        ZL(k_query<true>, div_up((size_t)ne * kQueryLanes, TB), TB, 0, st)(v, 1, ne, ebox.p, ebox.p, ecb.p, ecb.p, TE, big_e.p, (int)nbe, ne,
                                                     qcnt_ee.p, qoff_ee.p, ee.p);
    }
    if (nbp && n_pt)
        ZL(k_query_big<true>, nbp, 256, 0, st)(v, 0, big_p.p, pbox.p, tbox.p, nt, nullptr, qoff_pt.p, pt.p, pcb.p, tcb.p,
                                               TT, big_t.p, (int)nbt);
    if (nbq && n_ee)
        ZL(k_query_big<true>, nbq, 256, 0, st)(v, 1, big_q.p, ebox.p, ebox.p, ne, nullptr, qoff_ee.p, ee.p, ecb.p, ecb.p,
                                               TE, big_e.p, (int)nbe);
    ZLAUNCH();
}

}  // namespace zema
