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
    T* o = S_val + 9 * (size_t)S_diag[n];
    if (G.node_fixed[n]) {
        for (int i = 0; i < 9; ++i) o[i] = (i % 4 == 0) ? T(1) : T(0);
        return;
    }
    T m = (T)G.node_mass[n];
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
__global__ void k_seg_sum(const uint32_t* seg, uint32_t nu, const uint32_t* perm, const T* stage, T* out,
                          const uint64_t* key, uint64_t* ukey) {
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t u = (uint32_t)(gt >> 5);
    const int l = threadIdx.x & 31;
    if (u >= nu) return;  // the whole warp
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

// contact BSR: row pointers and columns from the unique (row, col) keys
__global__ void k_contact_rows(const uint64_t* ukey, uint32_t nu, int n_nodes, int* rowptr, int* col) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n_nodes) return;
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

__global__ void k_add_contact_grad(const uint64_t* ukey, const double* gsum, uint32_t nu, double* g) {
    uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nu) return;
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

template <class T>
__global__ void k_precond(Geo G, Bsr<T> S, Bsr<T> C, T* Minv_s, T* Minv_a) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= G.n_units) return;
    int kind = G.unit_kind[u], idx = G.unit_idx[u];
    if (kind == 0) {
        T a[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        add_row_blocks(S, idx, idx, idx + 1, a, 3, 0);
        add_row_blocks(C, idx, idx, idx + 1, a, 3, 0);
        inv3(a, Minv_s + 9 * (size_t)idx);
        return;
    }
    int n0 = G.aff_node0[idx];
    T A[144];
    for (int i = 0; i < 144; ++i) A[i] = 0;
    for (int j = 0; j < 4; ++j) {
        add_row_blocks(S, n0 + j, n0, n0 + 4, A, 12, 3 * j);
        add_row_blocks(C, n0 + j, n0, n0 + 4, A, 12, 3 * j);
    }
    // Gauss-Jordan inverse with partial pivoting (12x12, symmetric positive definite)
    T I[144];
    for (int i = 0; i < 144; ++i) I[i] = (i % 13 == 0) ? T(1) : T(0);
    for (int c = 0; c < 12; ++c) {
        int pv = c;
        for (int r = c + 1; r < 12; ++r)
            if (fabs(A[12 * r + c]) > fabs(A[12 * pv + c])) pv = r;
        if (pv != c)
            for (int j = 0; j < 12; ++j) {
                T t = A[12 * c + j];
                A[12 * c + j] = A[12 * pv + j];
                A[12 * pv + j] = t;
                t = I[12 * c + j];
                I[12 * c + j] = I[12 * pv + j];
                I[12 * pv + j] = t;
            }
        T ip = T(1) / A[12 * c + c];
        for (int j = 0; j < 12; ++j) {
            A[12 * c + j] *= ip;
            I[12 * c + j] *= ip;
        }
        for (int r = 0; r < 12; ++r) {
            if (r == c) continue;
            T f = A[12 * r + c];
            if (f == T(0)) continue;
            for (int j = 0; j < 12; ++j) {
                A[12 * r + j] -= f * A[12 * c + j];
                I[12 * r + j] -= f * I[12 * c + j];
            }
        }
    }
    for (int i = 0; i < 144; ++i) Minv_a[144 * (size_t)idx + i] = I[i];
}

// ---------------------------------------------------------------------------
// PCG with per-environment scalars.  Partial sums are kept per (env, chunk)
// and every block recombines them in the same order, so all blocks see the
// same alpha / beta and results are bit-reproducible.
// ---------------------------------------------------------------------------
struct PcgVec {
    double *x, *r, *z, *p, *q;
};

__device__ __forceinline__ double sum_chunks(const double* part, int env) {
    double s = 0.0;
    for (int c = 0; c < kChunks; ++c) s += part[(size_t)env * kChunks + c];
    return s;
}

template <class T>
__device__ __forceinline__ V3 spmv_row_warp(const Bsr<T>& A, int row, const double* p, int lane) {
    V3 y = v3(0, 0, 0);
    for (int k = A.rowptr[row] + lane; k < A.rowptr[row + 1]; k += 32) {
        const T* v = A.val + 9 * (size_t)k;
        V3 pc = ld3(p + 3 * (size_t)A.col[k]);
        y.x += (double)v[0] * pc.x + (double)v[1] * pc.y + (double)v[2] * pc.z;
        y.y += (double)v[3] * pc.x + (double)v[4] * pc.y + (double)v[5] * pc.z;
        y.z += (double)v[6] * pc.x + (double)v[7] * pc.y + (double)v[8] * pc.z;
    }
    return y;
}

// apply the preconditioner of a unit to r, write z; returns (r.z, r.r)
template <class T>
__device__ __forceinline__ void unit_precond(const Geo& G, int u, const T* Minv_s, const T* Minv_a,
                                             const double* r, double* z, double& rz, double& rr) {
    int kind = G.unit_kind[u], idx = G.unit_idx[u];
    rz = 0.0;
    rr = 0.0;
    if (kind == 0) {
        V3 rv = ld3(r + 3 * (size_t)idx);
        const T* M = Minv_s + 9 * (size_t)idx;
        double m[9];
        for (int q = 0; q < 9; ++q) m[q] = (double)M[q];
        V3 zv = v3(m[0] * rv.x + m[1] * rv.y + m[2] * rv.z, m[3] * rv.x + m[4] * rv.y + m[5] * rv.z,
                   m[6] * rv.x + m[7] * rv.y + m[8] * rv.z);
        st3(z + 3 * (size_t)idx, zv);
        rz = dot(rv, zv);
        rr = dot(rv, rv);
        return;
    }
    int n0 = G.aff_node0[idx];
    const T* M = Minv_a + 144 * (size_t)idx;
    const double* rb = r + 3 * (size_t)n0;
    for (int i = 0; i < 12; ++i) {
        double s = 0.0;
        for (int j = 0; j < 12; ++j) s += (double)M[12 * i + j] * rb[j];
        z[3 * (size_t)n0 + i] = s;
        rz += rb[i] * s;
        rr += rb[i] * rb[i];
    }
}

// ---------------------------------------------------------------------------
// Persistent PCG: one cooperative launch runs the whole solve.  Work is cut
// into tiles (contiguous units of one environment, a few each); blocks loop
// over tiles, write one partial sum per tile, and after each grid-wide
// barrier every block recombines the partials of each environment in tile
// order (identical in all blocks, so alpha, beta and the stop test agree
// everywhere and results are bit-reproducible).  Per env: the solve stops
// when |r| <= tol |b|; the launch ends when every env has stopped or after
// max_iter iterations.
// ---------------------------------------------------------------------------
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
    PcgVec V;
    const double* b;
    const Real* Minv_s;
    const Real* Minv_a;
    Tiles T;
    double* pt_rz;   // per-tile partials
    double* pt_rz2;
    double* pt_pq;
    double* pt_rr;
    double* pt_bb;
    int* conv;       // per env: in 1 = skip; out 1 = converged / skipped
    int* iters;      // per env
    double tol2;
    int max_iter;
};

// Sum of each env's tile partials into out[env].  Few envs: one warp per env,
// lanes stride over the tiles and a fixed shuffle tree combines them; many
// envs: one thread per env in tile order.  Every block computes identical
// values (same order).
__device__ __forceinline__ void env_sums(const Tiles& T, const double* part, int n_envs, double* out) {
    int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (n_envs <= nw * 4) {
        for (int e = w; e < n_envs; e += nw) {
            double s = 0.0;
            for (int t = T.env_start[e] + lane; t < T.env_start[e + 1]; t += 32) s += part[t];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) out[e] = s;
        }
    } else {
        for (int e = threadIdx.x; e < n_envs; e += blockDim.x) {
            double s = 0.0;
            for (int t = T.env_start[e]; t < T.env_start[e + 1]; ++t) s += part[t];
            out[e] = s;
        }
    }
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
    int* s_conv = (int*)(sm + 4 * NE);
    __shared__ double red[32];
    __shared__ int s_all;
    const Geo& G = a.G;
    PcgVec V = a.V;
    // init: x = 0, r = b, z = M^-1 r, p = z
    for (int t = blockIdx.x; t < a.T.n; t += gridDim.x) {
        int e = a.T.env[t];
        bool skip = a.conv[e] != 0;
        double rz = 0.0, bb = 0.0;
        if (!skip)
            for (int u = a.T.u0[t] + threadIdx.x; u < a.T.u1[t]; u += blockDim.x) {
                int kind = G.unit_kind[u], idx = G.unit_idx[u];
                int n0 = kind == 0 ? idx : G.aff_node0[idx], nn = kind == 0 ? 1 : 4;
                for (int j = 0; j < 3 * nn; ++j) {
                    size_t o = 3 * (size_t)n0 + j;
                    V.r[o] = a.b[o];
                    V.x[o] = 0.0;
                }
                double q1, q2;
                unit_precond(G, u, a.Minv_s, a.Minv_a, V.r, V.z, q1, q2);
                for (int j = 0; j < 3 * nn; ++j) V.p[3 * (size_t)n0 + j] = V.z[3 * (size_t)n0 + j];
                rz += q1;
                bb += q2;
            }
        double r1 = block_sum<256>(rz, red);
        double r2 = block_sum<256>(bb, red);
        if (threadIdx.x == 0) {
            a.pt_rz[t] = r1;
            a.pt_bb[t] = r2;
        }
    }
    grid.sync();
    env_sums(a.T, a.pt_rz, NE, s_rz);
    env_sums(a.T, a.pt_bb, NE, s_bb);
    __syncthreads();
    for (int e = threadIdx.x; e < NE; e += blockDim.x) s_conv[e] = a.conv[e] || !(s_bb[e] > 0.0);
    __syncthreads();
    int it = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            int all = 1;
            for (int e = 0; e < NE; ++e) all &= s_conv[e];
            s_all = all;
        }
        __syncthreads();
        if (s_all || it >= a.max_iter) break;
        // q = A p, partial p.q
        for (int t = blockIdx.x; t < a.T.n; t += gridDim.x) {
            int e = a.T.env[t];
            double s = 0.0;
            if (!s_conv[e]) {
                int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
                for (int n = a.T.n0[t] + w; n < a.T.n1[t]; n += blockDim.x >> 5) {
                    V3 y = spmv_row_warp(a.S, n, V.p, lane) + spmv_row_warp(a.C, n, V.p, lane);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        y.x += __shfl_xor_sync(0xffffffffu, y.x, o);
                        y.y += __shfl_xor_sync(0xffffffffu, y.y, o);
                        y.z += __shfl_xor_sync(0xffffffffu, y.z, o);
                    }
                    if (lane == 0) {
                        st3(V.q + 3 * (size_t)n, y);
                        s += dot(y, ld3(V.p + 3 * (size_t)n));
                    }
                }
            }
            double r1 = block_sum<256>(s, red);
            if (threadIdx.x == 0) a.pt_pq[t] = r1;
        }
        grid.sync();
        env_sums(a.T, a.pt_pq, NE, s_x);
        __syncthreads();
        // x += alpha p ; r -= alpha q ; z = M^-1 r ; partial r.z, r.r
        for (int t = blockIdx.x; t < a.T.n; t += gridDim.x) {
            int e = a.T.env[t];
            double rz = 0.0, rr = 0.0;
            if (!s_conv[e]) {
                double alpha = s_x[e] > 0.0 ? s_rz[e] / s_x[e] : 0.0;
                for (int u = a.T.u0[t] + threadIdx.x; u < a.T.u1[t]; u += blockDim.x) {
                    int kind = G.unit_kind[u], idx = G.unit_idx[u];
                    int n0 = kind == 0 ? idx : G.aff_node0[idx], nn = kind == 0 ? 1 : 4;
                    for (int j = 0; j < 3 * nn; ++j) {
                        size_t o = 3 * (size_t)n0 + j;
                        V.x[o] += alpha * V.p[o];
                        V.r[o] -= alpha * V.q[o];
                    }
                    double q1, q2;
                    unit_precond(G, u, a.Minv_s, a.Minv_a, V.r, V.z, q1, q2);
                    rz += q1;
                    rr += q2;
                }
            }
            double r1 = block_sum<256>(rz, red);
            double r2 = block_sum<256>(rr, red);
            if (threadIdx.x == 0) {
                a.pt_rz2[t] = r1;
                a.pt_rr[t] = r2;
            }
        }
        grid.sync();
        env_sums(a.T, a.pt_rz2, NE, s_x);
        env_sums(a.T, a.pt_rr, NE, s_y);
        __syncthreads();
        // beta, stop test, p = z + beta p
        for (int t = blockIdx.x; t < a.T.n; t += gridDim.x) {
            int e = a.T.env[t];
            if (s_conv[e] || !(s_y[e] > a.tol2 * s_bb[e])) continue;
            double beta = s_rz[e] != 0.0 ? s_x[e] / s_rz[e] : 0.0;
            for (int n = a.T.n0[t] + threadIdx.x; n < a.T.n1[t]; n += blockDim.x)
                for (int j = 0; j < 3; ++j) {
                    size_t o = 3 * (size_t)n + j;
                    V.p[o] = V.z[o] + beta * V.p[o];
                }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < NE; e += blockDim.x) {
            if (s_conv[e]) continue;
            if (blockIdx.x == 0) a.iters[e] += 1;
            if (!(s_y[e] > a.tol2 * s_bb[e])) s_conv[e] = 1;
            s_rz[e] = s_x[e];
        }
        ++it;
        grid.sync();
    }
    if (blockIdx.x == 0)
        for (int e = threadIdx.x; e < NE; e += blockDim.x) a.conv[e] = s_conv[e];
}

}  // namespace zema
