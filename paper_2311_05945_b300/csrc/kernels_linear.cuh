// Block-sparse assembly (3x3 blocks over nodes), block-Jacobi preconditioner
// and the PCG iteration with per-environment scalars.
#pragma once
#include <cooperative_groups.h>

#include "kernels_energy.cuh"

namespace zema {

// ---------------------------------------------------------------------------
// Static part: values of the fixed pattern, gathered per block from the tet
// and affine staging blocks in a fixed order (no atomics).
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_static_values(Geo G, int n_blocks, const T* stage, T* S_val) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_blocks) return;
    if (env_is_done(G, G.node_env[G.S_col[b]])) return;  // a block's nodes share one env
    T s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = G.S_src_ptr[b]; k < G.S_src_ptr[b + 1]; ++k) {
        const T* q = stage + 9 * (size_t)G.S_src[k];
        for (int i = 0; i < 9; ++i) s[i] += q[i];
    }
    for (int i = 0; i < 9; ++i) S_val[9 * (size_t)b + i] = s[i];
}

// diagonal blocks: + lumped mass (soft); fixed nodes become identity rows
template <class T>
__global__ void k_static_diag(Geo G, const int* S_diag, T* S_val) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.n_nodes) return;
    if (env_is_done(G, G.node_env[n])) return;
    T* o = S_val + 9 * (size_t)S_diag[n];
    if (G.node_fixed[n]) {
        for (int i = 0; i < 9; ++i) o[i] = (i % 4 == 0) ? T(1) : T(0);
        return;
    }
    double md = G.node_mass[n];
    if (md != 0.0 && G.spring_k) md += 2.0 * G.h * G.h * G.spring_k[n];  // spring: 2 h^2 k I
    T m = (T)md;
    o[0] += m;
    o[4] += m;
    o[8] += m;
}

// ---------------------------------------------------------------------------
// Contact part: each pair record (barrier or friction) with its 12x12
// stencil-space Hessian H and gradient g contributes node blocks
//   B(a, b) = sum_{k,l} W[a][k] W[b][l] H(k, l),  g(a) = sum_k W[a][k] g(k)
// over its distinct free nodes a, b (W: node weight in each stencil slot).
// ---------------------------------------------------------------------------
struct PairNodes {
    int m;
    int node[8];
    double W[8][4];
};

__device__ inline void pair_nodes(const Geo& G, const PairRec& r, PairNodes& P) {
    P.m = 0;
    for (int k = 0; k < 4; ++k) {
        int nd[4];
        double w[4];
        int c = sv_nodes(G, r.s[k], nd, w);
        for (int j = 0; j < c; ++j) {
            if (G.node_fixed[nd[j]]) continue;
            int a = 0;
            while (a < P.m && P.node[a] != nd[j]) ++a;
            if (a == P.m) {
                P.node[a] = nd[j];
                for (int q = 0; q < 4; ++q) P.W[a][q] = 0.0;
                ++P.m;
            }
            P.W[a][k] += w[j];
        }
    }
}

__global__ void k_contact_count(Geo G, const PairRec* rec, int n, uint32_t* cnt_blk, uint32_t* cnt_g) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (env_is_done(G, G.sv_env[rec[i].s[0]])) {  // a converged env: no blocks
        cnt_blk[i] = cnt_g[i] = 0;
        return;
    }
    PairNodes P;
    pair_nodes(G, rec[i], P);
    cnt_blk[i] = (uint32_t)(P.m * P.m);
    cnt_g[i] = (uint32_t)P.m;
}

// Per pair: its gradient per node and its m x m node blocks B_ab = sum_kl
// W[a][k] W[b][l] H_kl (slot Hessian blocks weighted by the nodes' slot
// weights), staged with their (row, col) keys.  kEmitPairLanes lanes per
// pair, each taking every kEmitPairLanes-th block.
constexpr int kEmitPairLanes = 8;
template <class T>
__global__ void k_contact_emit(Geo G, const PairRec* rec, int n, const T* pH, const double* pG,
                               const uint32_t* off_blk, const uint32_t* off_g, uint64_t* bkey, uint32_t* bval,
                               T* bstage, uint64_t* gkey, uint32_t* gval, double* gstage) {
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(gt / kEmitPairLanes), l = (int)(gt % kEmitPairLanes);
    if (i >= n) return;
    if (env_is_done(G, G.sv_env[rec[i].s[0]])) return;
    PairNodes P;
    pair_nodes(G, rec[i], P);
    const T* H = pH + (size_t)i * 144;
    const double* gg = pG + (size_t)i * 12;
    const uint32_t ob = off_blk[i], og = off_g[i];
    for (int a = l; a < P.m; a += kEmitPairLanes) {
        double s[3] = {0, 0, 0};
        for (int k = 0; k < 4; ++k) {
            double w = P.W[a][k];
            if (w == 0.0) continue;
            for (int r = 0; r < 3; ++r) s[r] += w * gg[3 * k + r];
        }
        uint32_t j = og + a;
        gkey[j] = (uint64_t)P.node[a];
        gval[j] = j;
        for (int r = 0; r < 3; ++r) gstage[3 * (size_t)j + r] = s[r];
    }
    for (int t = l; t < P.m * P.m; t += kEmitPairLanes) {
        const int a = t / P.m, b = t - a * P.m;
        T B[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = 0; k < 4; ++k) {
            T wa = (T)P.W[a][k];
            if (wa == T(0)) continue;
            for (int q = 0; q < 4; ++q) {
                T f = wa * (T)P.W[b][q];
                if (f == T(0)) continue;
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c) B[3 * r + c] += f * H[12 * (3 * k + r) + 3 * q + c];
            }
        }
        const uint32_t jb = ob + t;
        bkey[jb] = (uint64_t)P.node[a] * (uint64_t)G.n_nodes + (uint64_t)P.node[b];
        bval[jb] = jb;
        for (int q = 0; q < 9; ++q) bstage[9 * (size_t)jb + q] = B[q];
    }
}

// segment heads of a sorted key array
__global__ void k_heads(const uint64_t* key, uint32_t n, uint32_t* head) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    head[i] = (i == 0 || key[i] != key[i - 1]) ? 1u : 0u;
}

__global__ void k_seg_starts(const uint32_t* head, const uint32_t* hoff, uint32_t n, uint32_t* seg) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    if (i == n) {
        seg[hoff[n]] = n;
        return;
    }
    if (head[i]) seg[hoff[i]] = i;
}

// Sum the W-wide values of each unique key (deterministic).  One warp per
// key: lanes stride over the key's sorted segment and a fixed shuffle tree
// combines them, so the long segments (blocks between an affine body's nodes
// collect one contribution per pair touching the body) do not serialise.
template <int W, class T>
__device__ __forceinline__ void seg_sum_one(const uint32_t* seg, uint32_t u, int l, const uint32_t* perm,
                                            const T* stage, T* out, const uint64_t* key, uint64_t* ukey) {
    T s[W];
#pragma unroll
    for (int q = 0; q < W; ++q) s[q] = 0;
    const uint32_t b = seg[u], e = seg[u + 1];
    for (uint32_t i = b + l; i < e; i += 32) {
        const T* v = stage + (size_t)W * perm[i];
#pragma unroll
        for (int q = 0; q < W; ++q) s[q] += v[q];
    }
#pragma unroll
    for (int q = 0; q < W; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    }
    if (l < W) {
        T r = s[0];
#pragma unroll
        for (int q = 1; q < W; ++q) r = (l == q) ? s[q] : r;
        out[(size_t)W * u + l] = r;
    }
    if (l == 0) ukey[u] = key[b];
}

// The count of unique keys is read on the device (*nu_dev), so no host round
// trip sizes the launch: warps stride over the keys.
template <int W, class T>
__global__ void k_seg_sum(const uint32_t* seg, const uint32_t* nu_dev, const uint32_t* perm, const T* stage, T* out,
                          const uint64_t* key, uint64_t* ukey) {
    const uint32_t nu = *nu_dev;
    const int l = threadIdx.x & 31;
    const uint32_t n_warps = (uint32_t)((gridDim.x * (long long)blockDim.x) >> 5);
    for (uint32_t u = (uint32_t)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5); u < nu; u += n_warps)
        seg_sum_one<W, T>(seg, u, l, perm, stage, out, key, ukey);
}

// contact BSR: row pointers and columns from the unique (row, col) keys
__global__ void k_contact_rows(const uint64_t* ukey, const uint32_t* nu_dev, int n_nodes, int* rowptr, int* col) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n_nodes) return;
    const uint32_t nu = *nu_dev;
    // first unique key with row >= r
    uint64_t target = (uint64_t)r * (uint64_t)n_nodes;
    uint32_t lo = 0, hi = nu;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (ukey[mid] < target)
            lo = mid + 1;
        else
            hi = mid;
    }
    rowptr[r] = (int)lo;
    if (r < n_nodes)
        for (uint32_t k = lo; k < nu && ukey[k] < target + (uint64_t)n_nodes; ++k) col[k] = (int)(ukey[k] % n_nodes);
}

__global__ void k_add_contact_grad(const uint64_t* ukey, const double* gsum, const uint32_t* nu_dev, double* g) {
    uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= *nu_dev) return;
    size_t n = (size_t)ukey[u];
    for (int r = 0; r < 3; ++r) g[3 * n + r] += gsum[3 * (size_t)u + r];
}

// ---------------------------------------------------------------------------
// Block-Jacobi preconditioner: inverse 3x3 diagonal block per soft node,
// inverse 12x12 block per affine body.
// ---------------------------------------------------------------------------
template <class T>
struct Bsr {
    const int* rowptr;
    const int* col;
    const T* val;
};

template <class T>
__device__ __forceinline__ void add_row_blocks(const Bsr<T>& A, int row, int c0, int c1, T* out, int ld, int roff) {
    for (int k = A.rowptr[row]; k < A.rowptr[row + 1]; ++k) {
        int c = A.col[k];
        if (c < c0 || c >= c1) continue;
        const T* v = A.val + 9 * (size_t)k;
        int co = 3 * (c - c0);
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q) out[(roff + r) * ld + co + q] += v[3 * r + q];
    }
}

template <class T>
__device__ inline void inv3(const T* a, T* o) {
    T c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
    T det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    T id = T(1) / det;
    o[0] = c00 * id;
    o[3] = c01 * id;
    o[6] = c02 * id;
    o[1] = (a[2] * a[7] - a[1] * a[8]) * id;
    o[4] = (a[0] * a[8] - a[2] * a[6]) * id;
    o[7] = (a[1] * a[6] - a[0] * a[7]) * id;
    o[2] = (a[1] * a[5] - a[2] * a[4]) * id;
    o[5] = (a[2] * a[3] - a[0] * a[5]) * id;
    o[8] = (a[0] * a[4] - a[1] * a[3]) * id;
}

// Inverse 3x3 diagonal blocks of the soft units (one thread each); affine
// units are left to k_precond_aff.
template <class T>
__global__ void k_precond(Geo G, Bsr<T> S, Bsr<T> C, T* Minv_s) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= G.n_units) return;
    int kind = G.unit_kind[u], idx = G.unit_idx[u];
    if (kind != 0) return;
    if (env_is_done(G, G.node_env[idx])) return;
    T a[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    add_row_blocks(S, idx, idx, idx + 1, a, 3, 0);
    add_row_blocks(C, idx, idx, idx + 1, a, 3, 0);
    inv3(a, Minv_s + 9 * (size_t)idx);
}

// Blocks of row `row` whose columns lie in [c0, c1), for rows whose columns
// are sorted (the static pattern and the contact matrix both are): a binary
// search for c0, then at most c1 - c0 blocks.
template <class T>
__device__ __forceinline__ void add_row_blocks_sorted(const Bsr<T>& A, int row, int c0, int c1, T* out, int ld,
                                                      int roff) {
    int lo = A.rowptr[row], hi = A.rowptr[row + 1];
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (A.col[mid] < c0)
            lo = mid + 1;
        else
            hi = mid;
    }
    for (int k = lo, e = A.rowptr[row + 1]; k < e; ++k) {
        int c = A.col[k];
        if (c >= c1) break;
        const T* v = A.val + 9 * (size_t)k;
        int co = 3 * (c - c0);
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q) out[(roff + r) * ld + co + q] += v[3 * r + q];
    }
}

constexpr int kPrecondAffWarps = 4;  // affine bodies per CTA of k_precond_aff

// Inverse 12x12 diagonal block of every affine body: one warp per body,
// Gauss-Jordan with partial pivoting on [A | I].  Lane j < 24 holds column j
// of [A | I] (its 12 rows in registers); the pivot column's lane picks the
// pivot row, and the pivot value and the elimination factors (column c of
// each row) are broadcast by shuffles.  Pivot rule and arithmetic per entry
// are those of a serial Gauss-Jordan: row c scaled by 1 / pivot, then
// row r -= A[r][c] * row c for every r != c.
template <class T>
__global__ void __launch_bounds__(32 * kPrecondAffWarps) k_precond_aff(Geo G, Bsr<T> S, Bsr<T> C, T* Minv_a) {
    __shared__ double sbuf[kPrecondAffWarps * 144];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int idx = blockIdx.x * kPrecondAffWarps + w;
    if (idx >= G.n_aff) return;  // uniform over the warp
    if (env_is_done(G, G.node_env[G.aff_node0[idx]])) return;  // uniform over the warp
    T* sA = reinterpret_cast<T*>(sbuf) + 144 * w;
    for (int i = lane; i < 144; i += 32) sA[i] = T(0);
    __syncwarp();
    const int n0 = G.aff_node0[idx];
    if (lane < 4) {
        // row n0 + lane: static blocks, then contact blocks (the serial order)
        add_row_blocks_sorted(S, n0 + lane, n0, n0 + 4, sA, 12, 3 * lane);
        add_row_blocks_sorted(C, n0 + lane, n0, n0 + 4, sA, 12, 3 * lane);
    }
    __syncwarp();
    T a[12];
#pragma unroll
    for (int r = 0; r < 12; ++r)
        a[r] = lane < 12 ? sA[12 * r + lane] : (lane - 12 == r ? T(1) : T(0));
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        // pivot: largest |A[r][c]|, r >= c, first one on ties (lane c decides)
        int pv = c;
        T best = fabs(a[c]);
#pragma unroll
        for (int r = c + 1; r < 12; ++r)
            if (fabs(a[r]) > best) {
                best = fabs(a[r]);
                pv = r;
            }
        pv = __shfl_sync(0xffffffffu, pv, c);
#pragma unroll
        for (int r = c + 1; r < 12; ++r)
            if (r == pv) {
                T t = a[c];
                a[c] = a[r];
                a[r] = t;
            }
        const T ip = T(1) / __shfl_sync(0xffffffffu, a[c], c);
        a[c] *= ip;
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            if (r == c) continue;
            const T f = __shfl_sync(0xffffffffu, a[r], c);
            a[r] -= f * a[c];
        }
    }
    if (lane >= 12 && lane < 24) {
        T* o = Minv_a + 144 * (size_t)idx + (lane - 12);
#pragma unroll
        for (int r = 0; r < 12; ++r) o[12 * r] = a[r];
    }
}

// ---------------------------------------------------------------------------
// PCG with per-environment scalars.  Partial sums are kept per (env, chunk)
// and every block recombines them in the same order, so all blocks see the
// same alpha / beta and results are bit-reproducible.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Persistent PCG: one cooperative launch runs the whole solve (the path for
// envs too large for one cluster).  Work is cut into tiles: runs of soft
// units of one environment (sized at build so that there are a few tiles per
// SM), and one tile per affine body, whose four rows collect the contact
// blocks of every vertex touching the body and can be thousands of blocks
// long.  Blocks loop over tiles, write one partial sum per tile, and after
// each grid-wide barrier every block recombines the partials of each
// environment in tile order (identical in all blocks, so alpha, beta and the
// stop test agree everywhere and results are bit-reproducible).  Per env: the
// solve stops when |r| <= tol |b|, or on breakdown (p.Ap <= 0: x kept; a
// non-finite value marks the env with 2); the launch ends when every env has
// stopped or after max_iter iterations.
//
// The iteration runs in the matrix's type, its partial sums included (FP32 in
// the mixed form, where the caller refines the result against FP64
// residuals: B300's FP64 pipe is a small fraction of its FP32 rate, and
// FP64 tree sums over every tile in every block would cost more than the
// product itself).  Two grid barriers per iteration: the new direction
// p_k = z_k + beta p_{k-1} is formed on the fly inside the product (p
// double-buffered: the product reads p_{k-1} and z_k of its columns, the
// row's owner stores p_k), so a separate direction pass and its barrier are
// not needed.
// ---------------------------------------------------------------------------
constexpr int kPcgRowLanes = 4;  // lanes per soft row in the product

struct Tiles {
    int n;
    const int* u0;   // first unit of the tile
    const int* u1;
    const int* n0;   // node range of the tile's units
    const int* n1;
    const int* env;
    const int* env_start;  // n_envs + 1 tile offsets
};

template <class Real>
struct PcgArgs {
    Geo G;
    Bsr<Real> S, C;
    const double* b;   // right-hand side (FP64)
    double* x_out;     // solution (FP64)
    Real *x, *r, *z, *p, *p2, *q;  // work vectors, 3 n_nodes each
    const Real* Minv_s;
    const Real* Minv_a;
    Tiles T;
    Real* pt_rz;     // per-tile partials
    Real* pt_rz2;
    Real* pt_pq;
    Real* pt_rr;
    Real* pt_bb;
    int* conv;       // per env: in 1 = skip; out 1 = stopped, 2 = non-finite
    int* iters;      // per env
    double tol2;
    const double* tol2_env;  // per-env tolerance (squared, relative), or null
    int max_iter;
};

// Sum of each env's tile partials into out[env], identical in every block
// (same order).  Few envs: the whole block strides over an env's tiles and a
// fixed tree combines the threads; many envs: one thread per env in tile order.
// fixed-tree block sum in the solve's type (the result is valid in thread 0)
template <class Real>
__device__ __forceinline__ Real pcg_block_sum(Real v, Real* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    Real r = 0;
    if (w == 0) {
        r = l < (int)(blockDim.x >> 5) ? sh[l] : Real(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

template <class Real>
__device__ __forceinline__ void env_sums(const Tiles& T, const Real* part, int n_envs, double* out, Real* red) {
    if (n_envs <= 8) {
        for (int e = 0; e < n_envs; ++e) {
            Real s0 = 0, s1 = 0;
            const int t0 = T.env_start[e], t1 = T.env_start[e + 1];
            int t = t0 + threadIdx.x;
            for (; t + (int)blockDim.x < t1; t += 2 * blockDim.x) {
                s0 += __ldcg(part + t);
                s1 += __ldcg(part + t + blockDim.x);
            }
            if (t < t1) s0 += __ldcg(part + t);
            const Real v = pcg_block_sum<Real>(s0 + s1, red);
            if (threadIdx.x == 0) out[e] = (double)v;
        }
    } else {
        for (int e = threadIdx.x; e < n_envs; e += blockDim.x) {
            Real s = 0;
            for (int t = T.env_start[e]; t < T.env_start[e + 1]; ++t) s += __ldcg(part + t);
            out[e] = (double)s;
        }
    }
}

// env_sums of two partial arrays in one pass (the result pairs in outa, outb)
template <class Real>
__device__ __forceinline__ void env_sums2(const Tiles& T, const Real* pa, const Real* pb, int n_envs, double* outa,
                                          double* outb, Real* red) {
    if (n_envs <= 8) {
        for (int e = 0; e < n_envs; ++e) {
            Real sa = 0, sb = 0;
            for (int t = T.env_start[e] + threadIdx.x; t < T.env_start[e + 1]; t += blockDim.x) {
                sa += __ldcg(pa + t);
                sb += __ldcg(pb + t);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sa += __shfl_xor_sync(0xffffffffu, sa, o);
                sb += __shfl_xor_sync(0xffffffffu, sb, o);
            }
            const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
            if (l == 0) {
                red[w] = sa;
                red[nw + w] = sb;
            }
            __syncthreads();
            if (w == 0) {
                Real ra = l < nw ? red[l] : Real(0), rb = l < nw ? red[nw + l] : Real(0);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    ra += __shfl_xor_sync(0xffffffffu, ra, o);
                    rb += __shfl_xor_sync(0xffffffffu, rb, o);
                }
                if (l == 0) {
                    outa[e] = (double)ra;
                    outb[e] = (double)rb;
                }
            }
            __syncthreads();
        }
    } else {
        for (int e = threadIdx.x; e < n_envs; e += blockDim.x) {
            Real sa = 0, sb = 0;
            for (int t = T.env_start[e]; t < T.env_start[e + 1]; ++t) {
                sa += __ldcg(pa + t);
                sb += __ldcg(pb + t);
            }
            outa[e] = (double)sa;
            outb[e] = (double)sb;
        }
    }
}

// the tile is one affine body (its first node in n0)
__device__ __forceinline__ bool pcg_aff_tile(const Geo& G, const Tiles& T, int t) {
    const int u = T.u0[t];
    return T.u1[t] == u + 1 && G.unit_kind[u] == 1;
}

// component c of the direction at node n: z + beta p_old (beta = 0: z alone)
template <class Real>
__device__ __forceinline__ Real pcg_dir(const Real* z, const Real* pold, Real beta, size_t o) {
    Real v = z[o];
    if (beta != Real(0)) v += beta * pold[o];
    return v;
}

// blocks k0, k0 + step, ... < k1 of a row of A times the direction; four
// blocks per round so that their column and direction loads overlap
template <class Real>
__device__ __forceinline__ void pcg_row_part(const Bsr<Real>& A, int k0, int k1, int step, const Real* z,
                                             const Real* pold, Real beta, Real y[3]) {
    constexpr int U = 4;
    for (int k = k0; k < k1; k += U * step) {
        int c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) c[u] = k + u * step < k1 ? A.col[k + u * step] : -1;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (c[u] < 0) continue;
            const Real* v = A.val + 9 * (size_t)(k + u * step);
            const size_t o = 3 * (size_t)c[u];
            const Real p0 = pcg_dir(z, pold, beta, o), p1 = pcg_dir(z, pold, beta, o + 1),
                       p2 = pcg_dir(z, pold, beta, o + 2);
            y[0] += v[0] * p0 + v[1] * p1 + v[2] * p2;
            y[1] += v[3] * p0 + v[4] * p1 + v[5] * p2;
            y[2] += v[6] * p0 + v[7] * p1 + v[8] * p2;
        }
    }
}

// soft unit: z = M r on one node; returns r.z and r.r
template <class Real>
__device__ __forceinline__ void pcg_soft_precond(const Real* Minv_s, int n, const Real* r, Real* z, Real& rz,
                                                 Real& rr) {
    const Real* M = Minv_s + 9 * (size_t)n;
    const Real r0 = r[3 * (size_t)n], r1 = r[3 * (size_t)n + 1], r2 = r[3 * (size_t)n + 2];
    const Real z0 = M[0] * r0 + M[1] * r1 + M[2] * r2;
    const Real z1 = M[3] * r0 + M[4] * r1 + M[5] * r2;
    const Real z2 = M[6] * r0 + M[7] * r1 + M[8] * r2;
    z[3 * (size_t)n] = z0;
    z[3 * (size_t)n + 1] = z1;
    z[3 * (size_t)n + 2] = z2;
    rz += r0 * z0 + r1 * z1 + r2 * z2;
    rr += r0 * r0 + r1 * r1 + r2 * r2;
}

// affine unit, 12 threads: thread i computes row i of z = M r (12 x 12)
template <class Real>
__device__ __forceinline__ void pcg_aff_precond(const Real* Minv_a, int body, int n0, const Real* r, Real* z, int i,
                                                Real& rz, Real& rr) {
    const Real* M = Minv_a + 144 * (size_t)body;
    const Real* rb = r + 3 * (size_t)n0;
    Real zi = 0;
#pragma unroll
    for (int j = 0; j < 12; ++j) zi += M[12 * i + j] * rb[j];
    z[3 * (size_t)n0 + i] = zi;
    rz += rb[i] * zi;
    rr += rb[i] * rb[i];
}

template <class Real>
__global__ void __launch_bounds__(256) k_pcg_persistent(PcgArgs<Real> a) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    extern __shared__ double sm[];
    const int NE = a.G.n_envs;
    double* s_rz = sm;            // current r.z per env
    double* s_bb = sm + NE;       // b.b per env
    double* s_x = sm + 2 * NE;    // scratch per env (pq, then rz_new)
    double* s_y = sm + 3 * NE;    // scratch per env (rr)
    Real* s_alpha = reinterpret_cast<Real*>(sm + 4 * NE);  // this iteration's alpha per env
    Real* s_beta = s_alpha + NE;                             // beta of the next direction per env
    int* s_conv = reinterpret_cast<int*>(s_beta + NE);       // 0 running, 1 stopped, 2 non-finite
    __shared__ double red_d[32];
    Real* red = reinterpret_cast<Real*>(red_d);
    __shared__ int s_all;
    const Geo& G = a.G;
    const int tid = threadIdx.x;
    // init: x = 0, r = b, z = M^-1 r, previous direction 0
    for (int t = blockIdx.x; t < a.T.n; t += gridDim.x) {
        const int e = a.T.env[t];
        Real rz = 0, bb = 0;
        if (a.conv[e] == 0) {
            if (pcg_aff_tile(G, a.T, t)) {
                const int n0 = a.T.n0[t];
                if (tid < 12) {
                    const size_t o = 3 * (size_t)n0 + tid;
                    const Real bo = (Real)a.b[o];
                    a.r[o] = bo;
                    a.x[o] = Real(0);
                    a.p2[o] = Real(0);
                    bb = bo * bo;
                }
                __syncthreads();
                Real rr_unused = 0;
                if (tid < 12) pcg_aff_precond(a.Minv_a, G.unit_idx[a.T.u0[t]], n0, a.r, a.z, tid, rz, rr_unused);
            } else {
                for (int n = a.T.n0[t] + tid; n < a.T.n1[t]; n += blockDim.x) {
                    for (int c = 0; c < 3; ++c) {
                        const size_t o = 3 * (size_t)n + c;
                        const Real bo = (Real)a.b[o];
                        a.r[o] = bo;
                        a.x[o] = Real(0);
                        a.p2[o] = Real(0);
                        bb += bo * bo;
                    }
                    Real rr_unused = 0;
                    pcg_soft_precond(a.Minv_s, n, a.r, a.z, rz, rr_unused);
                }
            }
        }
        const Real r1 = pcg_block_sum<Real>(rz, red);
        const Real r2 = pcg_block_sum<Real>(bb, red);
        if (tid == 0) {
            a.pt_rz[t] = r1;
            a.pt_bb[t] = r2;
        }
    }
    grid.sync();
    env_sums(a.T, a.pt_rz, NE, s_rz, red);
    env_sums(a.T, a.pt_bb, NE, s_bb, red);
    __syncthreads();
    for (int e = tid; e < NE; e += blockDim.x) {
        const bool fin = isfinite(s_bb[e]) && isfinite(s_rz[e]);
        s_conv[e] = a.conv[e] ? 1 : (!fin ? 2 : (s_bb[e] > 0.0 ? 0 : 1));
        s_beta[e] = Real(0);
    }
    __syncthreads();
    Real* pold = a.p2;  // p_{k-1}
    Real* pcur = a.p;   // p_k, written this iteration
    const int sub = tid % kPcgRowLanes, grp = tid / kPcgRowLanes;
    const int rows_per_pass = blockDim.x / kPcgRowLanes;
    int it = 0;
    for (;;) {
        if (tid == 0) {
            int all = 1;
            for (int e = 0; e < NE; ++e) all &= s_conv[e] != 0;
            s_all = all;
        }
        __syncthreads();
        if (s_all || it >= a.max_iter) break;
        // p = z + beta p_old (own rows stored), q = A p, partial p.q
        for (int t = blockIdx.x; t < a.T.n; t += gridDim.x) {
            const int e = a.T.env[t];
            Real s = 0;
            if (!s_conv[e]) {
                const Real beta = s_beta[e];
                const int n0 = a.T.n0[t], n1 = a.T.n1[t];
                if (pcg_aff_tile(G, a.T, t)) {
                    // four long rows at once, 64 threads (two warps) each:
                    // strided partial products, a shuffle tree per warp,
                    // then the two warps of a row added in a fixed order
                    const int row = tid >> 6, l64 = tid & 63, w = tid >> 5;
                    const int n = n0 + row;
                    Real y[3] = {0, 0, 0};
                    if (n < n1) {
                        pcg_row_part(a.S, a.S.rowptr[n] + l64, a.S.rowptr[n + 1], 64, a.z, pold, beta, y);
                        pcg_row_part(a.C, a.C.rowptr[n] + l64, a.C.rowptr[n + 1], 64, a.z, pold, beta, y);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
                        for (int c = 0; c < 3; ++c) y[c] += __shfl_xor_sync(0xffffffffu, y[c], o);
                    if ((tid & 31) == 0)
                        for (int c = 0; c < 3; ++c) red[3 * w + c] = y[c];
                    __syncthreads();
                    if (l64 == 0 && n < n1) {
                        for (int c = 0; c < 3; ++c) {
                            const size_t o = 3 * (size_t)n + c;
                            const Real yc = red[3 * w + c] + red[3 * (w + 1) + c];
                            const Real pn = pcg_dir(a.z, pold, beta, o);
                            pcur[o] = pn;
                            a.q[o] = yc;
                            s += pn * yc;
                        }
                    }
                    __syncthreads();
                } else {
                    // soft rows: kPcgRowLanes lanes per row; the row loop is
                    // uniform over the block so every lane reaches the shuffles
                    for (int nb = n0; nb < n1; nb += rows_per_pass) {
                        const int n = nb + grp;
                        Real y[3] = {0, 0, 0};
                        if (n < n1) {
                            pcg_row_part(a.S, a.S.rowptr[n] + sub, a.S.rowptr[n + 1], kPcgRowLanes, a.z, pold, beta, y);
                            pcg_row_part(a.C, a.C.rowptr[n] + sub, a.C.rowptr[n + 1], kPcgRowLanes, a.z, pold, beta, y);
                        }
#pragma unroll
                        for (int o = kPcgRowLanes / 2; o > 0; o >>= 1)
                            for (int c = 0; c < 3; ++c) y[c] += __shfl_xor_sync(0xffffffffu, y[c], o);
                        if (n < n1 && sub == 0) {
                            Real d = 0;
                            for (int c = 0; c < 3; ++c) {
                                const size_t o = 3 * (size_t)n + c;
                                const Real pn = pcg_dir(a.z, pold, beta, o);
                                pcur[o] = pn;
                                a.q[o] = y[c];
                                d += pn * y[c];
                            }
                            s += d;
                        }
                    }
                }
            }
            const Real r1 = pcg_block_sum<Real>(s, red);
            if (tid == 0) a.pt_pq[t] = r1;
        }
        grid.sync();
        env_sums(a.T, a.pt_pq, NE, s_x, red);
        __syncthreads();
        // breakdown (p.Ap <= 0): stop with x kept; non-finite: mark the env;
        // otherwise alpha, once per env
        for (int e = tid; e < NE; e += blockDim.x) {
            if (s_conv[e]) continue;
            if (!(s_x[e] > 0.0))
                s_conv[e] = isfinite(s_x[e]) ? 1 : 2;
            else
                s_alpha[e] = (Real)(s_rz[e] / s_x[e]);
        }
        __syncthreads();
        // x += alpha p ; r -= alpha q ; z = M^-1 r ; partial r.z, r.r
        for (int t = blockIdx.x; t < a.T.n; t += gridDim.x) {
            const int e = a.T.env[t];
            Real rz = 0, rr = 0;
            if (!s_conv[e]) {
                const Real alpha = s_alpha[e];
                if (pcg_aff_tile(G, a.T, t)) {
                    const int n0 = a.T.n0[t];
                    if (tid < 12) {
                        const size_t o = 3 * (size_t)n0 + tid;
                        a.x[o] += alpha * pcur[o];
                        a.r[o] -= alpha * a.q[o];
                    }
                    __syncthreads();
                    if (tid < 12) pcg_aff_precond(a.Minv_a, G.unit_idx[a.T.u0[t]], n0, a.r, a.z, tid, rz, rr);
                } else {
                    for (int n = a.T.n0[t] + tid; n < a.T.n1[t]; n += blockDim.x) {
                        for (int c = 0; c < 3; ++c) {
                            const size_t o = 3 * (size_t)n + c;
                            a.x[o] += alpha * pcur[o];
                            a.r[o] -= alpha * a.q[o];
                        }
                        pcg_soft_precond(a.Minv_s, n, a.r, a.z, rz, rr);
                    }
                }
            }
            const Real r1 = pcg_block_sum<Real>(rz, red);
            const Real r2 = pcg_block_sum<Real>(rr, red);
            if (tid == 0) {
                a.pt_rz2[t] = r1;
                a.pt_rr[t] = r2;
            }
        }
        grid.sync();
        env_sums2(a.T, a.pt_rz2, a.pt_rr, NE, s_x, s_y, red);
        __syncthreads();
        // stop test and the next beta per env
        for (int e = tid; e < NE; e += blockDim.x) {
            if (s_conv[e]) continue;
            if (blockIdx.x == 0) a.iters[e] += 1;
            const double tol2 = a.tol2_env ? a.tol2_env[e] : a.tol2;
            if (!isfinite(s_y[e]) || !isfinite(s_x[e]))
                s_conv[e] = 2;
            else if (!(s_y[e] > tol2 * s_bb[e]))
                s_conv[e] = 1;
            s_beta[e] = (Real)(s_rz[e] != 0.0 ? s_x[e] / s_rz[e] : 0.0);
            s_rz[e] = s_x[e];
        }
        Real* tmp = pold;
        pold = pcur;
        pcur = tmp;
        ++it;
    }
    // x out in FP64 (envs that were skipped on entry are left untouched)
    for (int t = blockIdx.x; t < a.T.n; t += gridDim.x) {
        const int e = a.T.env[t];
        if (a.conv[e]) continue;
        for (int o = 3 * a.T.n0[t] + tid; o < 3 * a.T.n1[t]; o += blockDim.x) a.x_out[o] = (double)a.x[o];
    }
    grid.sync();
    if (blockIdx.x == 0)
        for (int e = tid; e < NE; e += blockDim.x) a.conv[e] = s_conv[e] == 2 ? 2 : (s_conv[e] ? 1 : 3);
}

}  // namespace zema
