// Block-Jacobi PCG with one thread-block cluster per environment.
//
// Each environment's system (a few thousand 3x3 block rows for the grasp
// workloads) is solved by the CTAs of one cluster.  A CTA owns a contiguous
// range of the env's soft-node rows, whose x, r and 3x3 preconditioner blocks
// stay in registers for the whole solve; the last CTA also owns the env's
// affine bodies (12x12 preconditioner rows in registers).  The rows of the
// affine bodies, whose contact blocks couple them to every soft node they
// touch, are split by block range across all CTAs of the cluster.  Every CTA
// holds the whole env's p in shared memory.  Per iteration:
//
//   stage    p_k = z_k + beta p_{k-1} in place over the env (z_k from L2,
//            written by its owner CTA), so the SpMV gathers p locally;
//   spmv     q = A p for the owned rows and the affine row shares, partial p.q;
//   B1       cluster barrier; every CTA sums the CTAs' partials in a fixed
//            order -> alpha (identical in all CTAs);
//   update   x += alpha p, r -= alpha q, z = M^-1 r on the owned units (the
//            affine rows' q: the CTAs' partials summed in rank order),
//            partial r.z and r.r;
//   B2       cluster barrier; sums -> beta and the stop test.
//
// Two hardware cluster barriers per iteration; inside the loop only z (one
// store per owned value, one L2 read per env value per CTA) and the matrix
// (read-only, L1/L2 resident) touch global memory;
// no grid-wide synchronisation and no atomics: results are bit-reproducible.
// Real is the arithmetic type of the whole solve, dot products and their
// cross-CTA sums included (double, or float in the mixed-precision mode: the
// stop tolerance, 1e-4 of |b|, is far above FP32 rounding, and B300's FP64
// rate is 1/64 of its FP32 rate).
#pragma once
#include <cooperative_groups.h>

#include "kernels_linear.cuh"

namespace zema {

template <class Real>
struct PcgcArgs {
    Geo G;
    Bsr<Real> S, C;
    const double* b;     // right-hand side, 3 per node
    double* x_out;       // solution, 3 per node (written for solved envs)
    Real* z;             // preconditioned residual, 3 per node (exchanged through L2)
    const Real* Minv_s;  // 9 per soft node
    const Real* Minv_a;  // 144 per affine body
    int* conv;           // per env in: 1 = skip; out: 1, or 2 after a non-finite value
    int* iters;          // per env: iterations run
    double tol2;
    const double* tol2_env;  // nullable: per-env |r|^2 / |b|^2 stop ratio instead of tol2
    int max_iter;
    int max_env_nodes;   // shared-memory layout bounds
    int max_rows;        // soft rows owned by one CTA, max over envs
    int max_aff;         // affine bodies per env, max over envs
    int slice_cap;       // blocks of a CTA's matrix slice that fit in shared memory (0: never staged)
    int chunk_cap;       // SpMV chunks a CTA can hold (more: one task per row instead)
    const int* env_list; // nullable: cluster k solves env env_list[k] (a group of envs), else env k
    const float4* pk;    // nullable (FP32 only): S then C packed by k_pack_blocks, read by unstaged CTAs
    int pk_c0;           // index of C's first block in pk
    // FP64 residual refinement inside the launch (FP32 solves): up to
    // `refine` rounds of r = b - A x in FP64 and, while |r|^2 > tol2 |b|^2,
    // a correction solve of A d = r added to x; 0 = none.  r64: 3 doubles
    // per node of scratch; refines (nullable): per env, the rounds taken
    int refine;
    double* r64;
    int* refines;
};

constexpr int kPcgcThreads = 512;
constexpr int kPcgcGroup = 4;   // lanes per row in the SpMV (8 rows per warp at a time)
constexpr int kPcgcMaxCluster = 16;
constexpr int kPcgcStageBatch = 16;  // values of z per thread whose loads are issued together
constexpr int kPcgcOwn = 2;         // soft rows per thread: a CTA owns at most 2 * kPcgcThreads rows
constexpr int kPcgcRefine = 3;      // FP64 residual refinements of an FP32 solve
constexpr int kPcgcRefAff = 16;     // affine bodies per env up to which the refinement runs in the launch
constexpr int kPcgcChunk = 8;       // blocks per SpMV chunk
constexpr int kPcgcRowIlp = 4;      // blocks per lane whose loads are issued together (matrix in L1/L2)
// values per node of the staged p vector
template <class Real>
__host__ __device__ constexpr int pcgc_pstride() {
    return 3;
}

__device__ __forceinline__ float ldcg_r(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg_r(const double* p) { return __ldcg(p); }

// All-reduce of K per-thread values over the cluster, in Real.  Each warp
// sums its lanes' values by shuffles into a slot of warp partials w; after a
// CTA barrier warp 0 sums the NW slots (a fixed shuffle tree), and lane l
// stores the CTA's K totals into slot rank of the reduction buffer of CTA l
// (distributed shared memory).  After the cluster barrier every thread sums
// the cs slots of its own copy in rank order, so all threads of all CTAs get
// the same bits.  One remote store per CTA pair and cs values to sum: the
// cluster barrier, not the traffic around it, sets the cost.  The cluster
// barrier also orders every CTA's earlier shared- and global-memory writes
// for the whole cluster.  red: K x kPcgcMaxCluster values; w: K x NW.
template <int K, class Real>
__device__ __forceinline__ void cluster_allreduce(cooperative_groups::cluster_group& cl, Real (&v)[K], Real* red,
                                                  Real* w_part, Real (&tot)[K]) {
    constexpr int NW = kPcgcThreads / 32;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int cs = (int)cl.num_blocks(), rank = (int)cl.block_rank();
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (l == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) w_part[k * NW + w] = v[k];
    __syncthreads();
    if (w == 0) {
        Real y[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            y[k] = l < NW ? w_part[k * NW + l] : Real(0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) y[k] += __shfl_xor_sync(0xffffffffu, y[k], o);
        }
        if (l < cs) {
            Real* dst = cl.map_shared_rank(red, l);
#pragma unroll
            for (int k = 0; k < K; ++k) dst[k * kPcgcMaxCluster + rank] = y[k];
        }
    }
    cl.sync();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        Real t = 0;
        for (int r = 0; r < cs; ++r) t += red[k * kPcgcMaxCluster + r];
        tot[k] = t;
    }
}

// q for one row: the blocks [s0, s1) of S followed by [c0, c1) of C, the 16
// lanes of a group striding over both ranges as one; p gathered from the
// staged env vector.  S and C are the global BSR arrays, or both the CTA's
// slice in shared memory (generic loads serve either).
template <class Real>
__device__ __forceinline__ void block_fma(const Bsr<Real>& S, const Bsr<Real>& C, int4 g, int ls, int j,
                                          const Real* s_p, int nb, int n_env, Real& y0, Real& y1, Real& y2) {
    constexpr int PS = pcgc_pstride<Real>();
    const bool in_s = j < ls;
    const int k = in_s ? g.x + j : g.z + (j - ls);
    const unsigned c = (unsigned)((in_s ? S.col : C.col)[k] - nb);
    if (c >= (unsigned)n_env) return;  // cannot happen: blocks stay inside one env
    const Real* v = (in_s ? S.val : C.val) + 9 * (size_t)k;
    const Real p0 = s_p[PS * c], p1 = s_p[PS * c + 1], p2 = s_p[PS * c + 2];
    y0 += v[0] * p0 + v[1] * p1 + v[2] * p2;
    y1 += v[3] * p0 + v[4] * p1 + v[5] * p2;
    y2 += v[6] * p0 + v[7] * p1 + v[8] * p2;
}

// a packed FP32 block: 12 floats (the 9 values, the column as int bits, 2
// pad) read as three 16-byte vectors, from the staged slice in shared memory
// or (kGlobal) from the packed matrix through the read-only data cache
template <bool kGlobal>
__device__ __forceinline__ void block_fma4(const float4* blk, const float* sp, int nb, int n_env, float& y0,
                                           float& y1, float& y2) {
    float4 a, b, c4;
    if constexpr (kGlobal) {
        a = __ldg(blk);
        b = __ldg(blk + 1);
        c4 = __ldg(blk + 2);
    } else {
        a = blk[0];
        b = blk[1];
        c4 = blk[2];
    }
    const unsigned c = (unsigned)(__float_as_int(c4.y) - nb);
    if (c >= (unsigned)n_env) return;  // cannot happen: blocks stay inside one env
    const float p0 = sp[3 * c], p1 = sp[3 * c + 1], p2 = sp[3 * c + 2];
    y0 += a.x * p0 + a.y * p1 + a.z * p2;
    y1 += a.w * p0 + b.x * p1 + b.y * p2;
    y2 += b.z * p0 + b.w * p1 + c4.x * p2;
}

// blocks [jb, je) of a row of packed blocks (S range, then C range)
template <bool kGlobal>
__device__ __forceinline__ void row_part4(const float4* slice, int4 g, int jb, int je, const float* sp, int nb,
                                          int n_env, int gl, float& y0, float& y1, float& y2) {
    // the accumulation order of row_part (kPcgcRowIlp accumulators summed in
    // order), so that a staged and an unstaged slice give the same bits
    const int ls = g.y - g.x;
    float a[kPcgcRowIlp][3];
#pragma unroll
    for (int t = 0; t < kPcgcRowIlp; ++t) a[t][0] = a[t][1] = a[t][2] = 0.0f;
    for (int j0 = jb + gl; j0 < je; j0 += kPcgcRowIlp * kPcgcGroup) {
#pragma unroll
        for (int t = 0; t < kPcgcRowIlp; ++t) {
            const int j = j0 + t * kPcgcGroup;
            if (j < je)
                block_fma4<kGlobal>(slice + 3 * (size_t)(j < ls ? g.x + j : g.z + (j - ls)), sp, nb, n_env, a[t][0], a[t][1],
                           a[t][2]);
        }
    }
#pragma unroll
    for (int t = 0; t < kPcgcRowIlp; ++t) {
        y0 += a[t][0];
        y1 += a[t][1];
        y2 += a[t][2];
    }
}

// blocks [jb, je) of the row's combined index space (S range, then C range)
template <class Real>
__device__ __forceinline__ void row_part(const Bsr<Real>& S, const Bsr<Real>& C, int4 g, int jb, int je,
                                         const Real* s_p, int nb, int n_env, int gl, Real& y0, Real& y1, Real& y2) {
    const int ls = g.y - g.x, n = je;
    // kPcgcRowIlp blocks per lane per pass (predicated, independent
    // accumulators) so that their loads from L1/L2 are in flight together;
    // the accumulators are summed in a fixed order
    Real a[kPcgcRowIlp][3];
#pragma unroll
    for (int t = 0; t < kPcgcRowIlp; ++t) a[t][0] = a[t][1] = a[t][2] = Real(0);
    for (int j0 = jb + gl; j0 < n; j0 += kPcgcRowIlp * kPcgcGroup) {
#pragma unroll
        for (int t = 0; t < kPcgcRowIlp; ++t) {
            const int j = j0 + t * kPcgcGroup;
            if (j < n) block_fma(S, C, g, ls, j, s_p, nb, n_env, a[t][0], a[t][1], a[t][2]);
        }
    }
#pragma unroll
    for (int t = 0; t < kPcgcRowIlp; ++t) {
        y0 += a[t][0];
        y1 += a[t][1];
        y2 += a[t][2];
    }
}

template <class Real>
__device__ __forceinline__ Real group_sum(Real v) {
#pragma unroll
    for (int o = kPcgcGroup / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// FP64 products of the blocks [jb, je) of a task's combined range (S, then
// C) with the FP64 vector xg (global, written earlier in this launch: read
// through L2), the matrix from the staged slice, the packed FP32 matrix or
// the BSR arrays, as the SpMV reads it
template <class Real>
__device__ __forceinline__ void row_part64(const PcgcArgs<Real>& a, bool staged, const float* smv, int4 g, int jb,
                                           int je, const double* xg, int gl, double& y0, double& y1, double& y2) {
    const int ls = g.y - g.x;
    for (int j = jb + gl; j < je; j += kPcgcGroup) {
        const bool in_s = j < ls;
        double v[9];
        int col;
        if (staged) {
            const int k = in_s ? g.x + j : g.z + (j - ls);
            const float* r = smv + 12 * (size_t)k;
#pragma unroll
            for (int c = 0; c < 9; ++c) v[c] = r[c];
            col = __float_as_int(r[9]);
        } else if (a.pk) {
            const int k = in_s ? g.x + j : a.pk_c0 + g.z + (j - ls);
            const float4 q0 = __ldg(a.pk + 3 * (size_t)k), q1 = __ldg(a.pk + 3 * (size_t)k + 1),
                         q2 = __ldg(a.pk + 3 * (size_t)k + 2);
            v[0] = q0.x, v[1] = q0.y, v[2] = q0.z, v[3] = q0.w, v[4] = q1.x, v[5] = q1.y, v[6] = q1.z, v[7] = q1.w;
            v[8] = q2.x;
            col = __float_as_int(q2.y);
        } else {
            const int k = in_s ? g.x + j : g.z + (j - ls);
            const Real* r = (in_s ? a.S.val : a.C.val) + 9 * (size_t)k;
#pragma unroll
            for (int c = 0; c < 9; ++c) v[c] = (double)r[c];
            col = (in_s ? a.S.col : a.C.col)[k];
        }
        const double x0 = __ldcg(xg + 3 * (size_t)col), x1 = __ldcg(xg + 3 * (size_t)col + 1),
                     x2 = __ldcg(xg + 3 * (size_t)col + 2);
        y0 += v[0] * x0 + v[1] * x1 + v[2] * x2;
        y1 += v[3] * x0 + v[4] * x1 + v[5] * x2;
        y2 += v[6] * x0 + v[7] * x1 + v[8] * x2;
    }
}

// kMinBlocks CTAs resident per SM: 1 keeps every owned row's state in
// registers and may stage the matrix slice in shared memory (few envs); 2
// halves the register budget (the compiler spills the preconditioner blocks
// to L1-cached local memory) and never stages, so that twice as many
// clusters run at once (many envs, where the solve is latency-bound)
template <class Real, int kMinBlocks>
__global__ void __launch_bounds__(kPcgcThreads, kMinBlocks) k_pcg_cluster(PcgcArgs<Real> a) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const Geo& G = a.G;
    const int cs = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int e = a.env_list ? a.env_list[blockIdx.x / cs] : (int)(blockIdx.x / cs);
    if (e >= G.n_envs) return;       // whole cluster (grid is n_envs * cs)
    if (a.conv[e] != 0) return;      // whole cluster: env needs no solve

    constexpr int NW = kPcgcThreads / 32;
    extern __shared__ int4 smi[];
    const int max_tasks = a.max_rows + 4 * a.max_aff;
    int4* s_rng = smi;                         // [max_tasks] block ranges of the SpMV tasks in S and C
    int4* s_chunk = s_rng + max_tasks;         // [chunk_cap] (task, first, end) of each SpMV chunk
    int* s_cpre = (int*)(s_chunk + a.chunk_cap);  // [max_tasks + 1] first chunk of each task
    Real* s_w = (Real*)(s_cpre + ((max_tasks + 4) & ~3));  // [3][NW] warp partials of the all-reduce
    Real* s_part = s_w + 3 * NW;       // [4] this CTA's partials (read by the cluster)
    Real* s_tot = s_part + 4;          // [4] cluster totals
    constexpr int PS = pcgc_pstride<Real>();
    Real* s_p = s_tot + 4;             // [PS * max_env_nodes] p over the whole env (16-byte aligned)
    Real* s_q = s_p + PS * (size_t)a.max_env_nodes;  // [3 * max_rows] q of the owned soft rows
    Real* s_qa = s_q + 3 * (size_t)a.max_rows;      // [12 * max_aff] partial q of the affine rows
    Real* s_ra = s_qa + 12 * (size_t)a.max_aff;     // [12 * max_aff] r of the affine rows (last rank)
    Real* s_cpart = s_ra + 12 * (size_t)a.max_aff;  // [3 * chunk_cap] SpMV chunk partial products
    // [12 * slice_cap] this CTA's matrix blocks (S then C), FP32 only, 16-byte aligned
    float* s_mval = (float*)(((uintptr_t)(s_cpart + 3 * (size_t)a.chunk_cap) + 15) & ~(uintptr_t)15);
    __shared__ int s_staged;
    // reduction buffers of cluster_allreduce: [0] the p.q sum, [1] the r.z
    // and r.r sums (alternating uses never overlap: see the hazard note at
    // the loop)
    __shared__ Real s_red[2][2 * kPcgcMaxCluster];
    Real* zw = a.z;                                 // z, 3 per node, in global memory
    const Real* __restrict__ zg = a.z;

    const int nb = G.env_node_start[e], nend = G.env_node_start[e + 1], n_env = nend - nb;
    const int ab0 = G.env_aff_start[e], n_aff = G.env_aff_start[e + 1] - ab0;
    const int ns1 = n_aff ? G.aff_node0[ab0] : nend;  // soft nodes are [nb, ns1), affine nodes [ns1, nend)
    const int n_soft = ns1 - nb, n_arow = nend - ns1;
    // soft rows per CTA, balanced by the rows' stored blocks (static and
    // contact, plus 2 per row for its fixed cost) when no CTA then owns more
    // than twice its equal share (and no more than the layout's max_rows),
    // else an equal split; every CTA finds the same boundaries (binary
    // searches over the same prefix sums).  The bound depends on this env
    // alone, so the partition does too.
    __shared__ int s_bounds[kPcgcMaxCluster + 1];
    if (threadIdx.x == 0) {
        const int max_rows_env = min(2 * ((n_soft + cs - 1) / cs) + 1, a.max_rows);
        auto cum = [&](int row) -> long long {
            return (long long)a.S.rowptr[row] + a.C.rowptr[row] + 2ll * row;
        };
        const long long c0 = cum(nb), tot = cum(ns1) - c0;
        bool ok = true;
        s_bounds[0] = nb;
        for (int r = 1; r <= cs; ++r) {
            int b = ns1;
            if (r < cs) {
                const long long target = (tot * r) / cs;
                int l = s_bounds[r - 1], h = ns1;  // first row with cum - c0 >= target
                while (l < h) {
                    const int m = (l + h) >> 1;
                    if (cum(m) - c0 < target)
                        l = m + 1;
                    else
                        h = m;
                }
                b = l;
            }
            s_bounds[r] = b;
            ok &= b - s_bounds[r - 1] <= max_rows_env - 1;
        }
        if (!ok)
            for (int r = 0; r <= cs; ++r) s_bounds[r] = nb + (int)(((long long)n_soft * r) / cs);
    }
    __syncthreads();
    const int lo = s_bounds[rank], hi = s_bounds[rank + 1];
    const int n_own = hi - lo;
    const bool aff_owner = rank == cs - 1;
    const int tid = threadIdx.x;
    // thread tid owns soft nodes lo + tid + j * kPcgcThreads (j < kPcgcOwn) and,
    // in the last rank, component tid of the affine rows (tid < 12 n_aff)
    const bool own_a = aff_owner && tid < 12 * n_aff;

    // the 3x3 blocks of M^-1 of the owned rows, and the affine owner's rows
    // of its bodies' 12x12 blocks, stay in registers for the whole launch
    Real xs[kPcgcOwn][3], rs[kPcgcOwn][3], Ms[kPcgcOwn][9];
    Real xa = 0, ra = 0, Ma[12];
#pragma unroll
    for (int j = 0; j < kPcgcOwn; ++j) {
        const int i = tid + j * kPcgcThreads;
        if (i >= n_own) continue;
        const Real* M = a.Minv_s + 9 * (size_t)(lo + i);
#pragma unroll
        for (int c = 0; c < 9; ++c) Ms[j][c] = M[c];
    }
    if (own_a) {
        const int bi = tid / 12, i = tid - 12 * bi;
        const Real* M = a.Minv_a + 144 * (size_t)(ab0 + bi) + 12 * i;
#pragma unroll
        for (int c = 0; c < 12; ++c) Ma[c] = M[c];
    }
    // ---- init of a solve from the right-hand side rhs (b, or the FP64
    // residual of a refinement round): x = 0, r = rhs, z = M^-1 r (x and r
    // stay in registers); the thread's share of r.z and r.r into acc
    auto init = [&](const double* rhs, Real (&acc)[2]) {
        acc[0] = acc[1] = 0;
#pragma unroll
        for (int j = 0; j < kPcgcOwn; ++j) {
            const int i = tid + j * kPcgcThreads;
            if (i >= n_own) continue;
            const size_t o = 3 * (size_t)(lo + i);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                rs[j][c] = (Real)rhs[o + c];
                xs[j][c] = 0;
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Real z = Ms[j][3 * c] * rs[j][0] + Ms[j][3 * c + 1] * rs[j][1] + Ms[j][3 * c + 2] * rs[j][2];
                zw[3 * (size_t)(lo + i) + c] = z;
                acc[0] += rs[j][c] * z;
                acc[1] += rs[j][c] * rs[j][c];
            }
        }
        xa = 0;
        if (own_a) {
            ra = (Real)rhs[3 * (size_t)ns1 + tid];
            s_ra[tid] = ra;
        }
        __syncthreads();
        if (own_a) {
            const int bi = tid / 12;
            Real z = 0;
#pragma unroll
            for (int c = 0; c < 12; ++c) z += Ma[c] * s_ra[12 * bi + c];
            zw[3 * (size_t)ns1 + tid] = z;
            acc[0] += ra * z;
            acc[1] += ra * ra;
        }
    };
    Real acc0[2];
    init(a.b, acc0);
    // block ranges of this CTA's SpMV tasks (fixed for the solve)
    const int n_tasks = n_own + n_arow;
    for (int task = tid; task < n_tasks; task += kPcgcThreads) {
        int4 g;
        if (task < n_own) {
            int row = lo + task;
            g = make_int4(a.S.rowptr[row], a.S.rowptr[row + 1], a.C.rowptr[row], a.C.rowptr[row + 1]);
        } else {
            int row = ns1 + (task - n_own);
            int k0 = a.S.rowptr[row], len = a.S.rowptr[row + 1] - k0;
            int c0 = a.C.rowptr[row], clen = a.C.rowptr[row + 1] - c0;
            g = make_int4(k0 + (int)(((long long)len * rank) / cs), k0 + (int)(((long long)len * (rank + 1)) / cs),
                          c0 + (int)(((long long)clen * rank) / cs), c0 + (int)(((long long)clen * (rank + 1)) / cs));
        }
        s_rng[task] = g;
    }
    // the CTA's matrix slice (fixed during the solve) into shared memory when
    // it fits: the soft rows' S and C ranges are contiguous, the affine row
    // shares follow; s_rng then holds offsets into the staged arrays
    __syncthreads();
    const int S0 = a.S.rowptr[lo], nS = a.S.rowptr[hi] - S0;
    const int C0 = a.C.rowptr[lo], nC = a.C.rowptr[hi] - C0;
    if (tid == 0) {
        long long tot = (long long)nS + nC;
        for (int t = n_own; t < n_tasks; ++t) tot += (s_rng[t].y - s_rng[t].x) + (s_rng[t].w - s_rng[t].z);
        s_staged = tot <= a.slice_cap ? 1 : 0;
    }
    __syncthreads();
    const bool staged = s_staged != 0;
    if (staged) {
        // block b of the slice: 12 floats, values at 12 b + 0..8, column at 12 b + 9
        auto put = [&](const Bsr<Real>& M, int k0, int n, int off) {
            for (int i = tid; i < 9 * n; i += kPcgcThreads) {
                const int b = i / 9;
                s_mval[12 * (size_t)(off + b) + (i - 9 * b)] = (float)M.val[9 * (size_t)k0 + i];
            }
            for (int i = tid; i < n; i += kPcgcThreads) {
                s_mval[12 * (size_t)(off + i) + 9] = __int_as_float(M.col[k0 + i]);
                s_mval[12 * (size_t)(off + i) + 10] = 0.0f;
                s_mval[12 * (size_t)(off + i) + 11] = 0.0f;
            }
        };
        put(a.S, S0, nS, 0);
        put(a.C, C0, nC, nS);
        // affine shares, in task order after the soft rows' blocks
        int off = nS + nC;
        for (int t = n_own; t < n_tasks; ++t) {
            const int4 g = s_rng[t];
            const int ls = g.y - g.x, lc = g.w - g.z;
            put(a.S, g.x, ls, off);
            put(a.C, g.z, lc, off + ls);
            off += ls + lc;
        }
        __syncthreads();
        // ranges into the staged arrays (S part, then C part of the same arrays)
        for (int task = tid; task < n_own; task += kPcgcThreads) {
            const int row = lo + task;
            s_rng[task] = make_int4(a.S.rowptr[row] - S0, a.S.rowptr[row + 1] - S0, nS + a.C.rowptr[row] - C0,
                                    nS + a.C.rowptr[row + 1] - C0);
        }
        if (tid == 0) {
            int o = nS + nC;
            for (int t = n_own; t < n_tasks; ++t) {
                const int4 g = s_rng[t];
                const int ls = g.y - g.x, lc = g.w - g.z;
                s_rng[t] = make_int4(o, o + ls, o + ls, o + ls + lc);
                o += ls + lc;
            }
        }
    }
    const float4* slice4 = reinterpret_cast<const float4*>(s_mval);
    const float* sp4 = reinterpret_cast<const float*>(s_p);
    // SpMV work in chunks of at most kPcgcChunk blocks, spread over all lane
    // groups whatever the row lengths; each row's chunk products are summed
    // in chunk order afterwards
    __shared__ int s_nchunks;
    __syncthreads();
    if (tid == 0) {
        int c = 0;
        for (int t = 0; t < n_tasks; ++t) {
            const int4 g = s_rng[t];
            const int len = (g.y - g.x) + (g.w - g.z);
            s_cpre[t] = c;
            c += len > 0 ? (len + kPcgcChunk - 1) / kPcgcChunk : 1;
        }
        s_cpre[n_tasks] = c;
        s_nchunks = c;
    }
    __syncthreads();
    const int n_chunks = s_nchunks;
    const bool chunked = n_chunks <= a.chunk_cap;
    if (chunked)
        for (int t = tid; t < n_tasks; t += kPcgcThreads) {
            const int4 g = s_rng[t];
            const int len = (g.y - g.x) + (g.w - g.z);
            for (int c = s_cpre[t], j = 0; c < s_cpre[t + 1]; ++c, j += kPcgcChunk)
                s_chunk[c] = make_int4(t, j, min(len, j + kPcgcChunk), 0);
        }
    constexpr int kGroupsPerWarp = 32 / kPcgcGroup;
    const int warp = tid >> 5, sub = (tid & 31) / kPcgcGroup, gl = tid & (kPcgcGroup - 1);
    const int n_groups = kPcgcThreads / kPcgcGroup;
    // FP64 reductions and affine partial products of the refinement rounds
    __shared__ double s_red64[2 * kPcgcMaxCluster];
    __shared__ double s_w64[2 * NW];
    __shared__ double s_qa64[12 * kPcgcRefAff];
    Real tol_pass = (Real)(a.tol2_env ? a.tol2_env[e] : a.tol2);
    int it_total = 0, n_ref = 0, status = 3;
    for (int pass = 0;; ++pass) {
    // the all-reduce's cluster barrier also orders s_rng, the chunks and the
    // staged slice within the CTA (and, in later passes, z of the new init)
    Real t0[2];
    cluster_allreduce<2>(cl, acc0, s_red[1], s_w, t0);  // r.z, r.r
    Real rz = t0[0];
    const Real bb = t0[1];
    const Real stop2 = tol_pass * bb;
    bool bad = !isfinite(bb);
    bool done = bad || !(bb > Real(0));
    Real beta = 0;
    int it = 0;
    while (!done && it < a.max_iter) {
        // ---- p_k = z_k + beta p_{k-1} over the env, in place (every CTA
        // holds the same p); z comes from L2, written there by its owner
        // (the env's 3 n_env values as one flat range: kPcgcStageBatch
        // independent loads per thread, one L2 round trip for small envs)
        const int n3e = 3 * n_env;
        const Real* __restrict__ zs = zg + 3 * (size_t)nb;
        for (int i0 = tid; i0 < n3e; i0 += kPcgcStageBatch * kPcgcThreads) {
            Real zv[kPcgcStageBatch];
#pragma unroll
            for (int j = 0; j < kPcgcStageBatch; ++j) {
                const int i = i0 + j * kPcgcThreads;
                zv[j] = ldcg_r(zs + (i < n3e ? i : 0));
            }
#pragma unroll
            for (int j = 0; j < kPcgcStageBatch; ++j) {
                const int i = i0 + j * kPcgcThreads;
                if (i < n3e) s_p[i] = it > 0 ? zv[j] + beta * s_p[i] : zv[j];
            }
        }
        __syncthreads();
        // ---- q = A p: owned soft rows, then this CTA's share of each affine row
        Real pq[1] = {0};
        // kGroupsPerWarp groups of kPcgcGroup lanes per warp; the loops are
        // uniform over the warp so that every lane takes part in the shuffles
        if (chunked) {
            for (int c0 = kGroupsPerWarp * warp; c0 < n_chunks; c0 += n_groups) {
                const int ci = c0 + sub;
                const bool valid = ci < n_chunks;
                Real y0 = 0, y1 = 0, y2 = 0;
                if (valid) {
                    const int4 ch = s_chunk[ci];
                    const int4 g = s_rng[ch.x];
                    if constexpr (sizeof(Real) == sizeof(float)) {
                        if (staged)
                            row_part4<false>(slice4, g, ch.y, ch.z, sp4, nb, n_env, gl, y0, y1, y2);
                        else if (a.pk)
                            row_part4<true>(a.pk, make_int4(g.x, g.y, g.z + a.pk_c0, g.w + a.pk_c0), ch.y, ch.z, sp4,
                                            nb, n_env, gl, y0, y1, y2);
                        else
                            row_part(a.S, a.C, g, ch.y, ch.z, s_p, nb, n_env, gl, y0, y1, y2);
                    } else {
                        row_part(a.S, a.C, g, ch.y, ch.z, s_p, nb, n_env, gl, y0, y1, y2);
                    }
                }
                y0 = group_sum(y0);
                y1 = group_sum(y1);
                y2 = group_sum(y2);
                if (valid && gl == 0) {
                    s_cpart[3 * ci] = y0;
                    s_cpart[3 * ci + 1] = y1;
                    s_cpart[3 * ci + 2] = y2;
                }
            }
            __syncthreads();
            for (int t = tid; t < n_tasks; t += kPcgcThreads) {
                Real y0 = 0, y1 = 0, y2 = 0;
                for (int c = s_cpre[t]; c < s_cpre[t + 1]; ++c) {
                    y0 += s_cpart[3 * c];
                    y1 += s_cpart[3 * c + 1];
                    y2 += s_cpart[3 * c + 2];
                }
                const int row = t < n_own ? lo + t : ns1 + (t - n_own);
                Real* qd = t < n_own ? s_q + 3 * t : s_qa + 3 * (t - n_own);
                qd[0] = y0;
                qd[1] = y1;
                qd[2] = y2;
                const Real* pr = s_p + PS * (row - nb);
                pq[0] += pr[0] * y0 + pr[1] * y1 + pr[2] * y2;
            }
        } else
        for (int t0 = kGroupsPerWarp * warp; t0 < n_tasks; t0 += n_groups) {
            const int task = t0 + sub;
            const bool valid = task < n_tasks;
            Real y0 = 0, y1 = 0, y2 = 0;
            int row = 0;
            if (valid) {
                int4 g = s_rng[task];
                row = task < n_own ? lo + task : ns1 + (task - n_own);
                const int len = (g.y - g.x) + (g.w - g.z);
                if constexpr (sizeof(Real) == sizeof(float)) {
                    if (staged)
                        row_part4<false>(slice4, g, 0, len, sp4, nb, n_env, gl, y0, y1, y2);
                    else if (a.pk)
                        row_part4<true>(a.pk, make_int4(g.x, g.y, g.z + a.pk_c0, g.w + a.pk_c0), 0, len, sp4, nb,
                                        n_env, gl, y0, y1, y2);
                    else
                        row_part(a.S, a.C, g, 0, len, s_p, nb, n_env, gl, y0, y1, y2);
                } else {
                    row_part(a.S, a.C, g, 0, len, s_p, nb, n_env, gl, y0, y1, y2);
                }
            }
            y0 = group_sum(y0);
            y1 = group_sum(y1);
            y2 = group_sum(y2);
            if (valid && gl == 0) {
                Real* qd = task < n_own ? s_q + 3 * task : s_qa + 3 * (task - n_own);
                qd[0] = y0;
                qd[1] = y1;
                qd[2] = y2;
                const Real* pr = s_p + PS * (row - nb);
                pq[0] += pr[0] * y0 + pr[1] * y1 + pr[2] * y2;
            }
        }
        // B1.  Hazard note: a CTA writes buffer 0 again only after passing
        // B2, which every CTA reaches after reading buffer 0; likewise
        // buffer 1 between B2 and the next B1
        Real t1[1];
        cluster_allreduce<1>(cl, pq, s_red[0], s_w, t1);
        const Real pqt = t1[0];
        if (!(pqt > Real(0))) {  // breakdown: keep x and stop (same in all CTAs); non-finite is an error
            bad = !isfinite(pqt);
            break;
        }
        const Real alpha = rz / pqt;
        // ---- x += alpha p, r -= alpha q, z = M^-1 r on the owned units
        Real acc[2] = {0, 0};
#pragma unroll
        for (int j = 0; j < kPcgcOwn; ++j) {
            const int i = tid + j * kPcgcThreads;
            if (i >= n_own) continue;
            const Real* pr = s_p + PS * (lo + i - nb);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xs[j][c] += alpha * pr[c];
                rs[j][c] -= alpha * s_q[3 * i + c];
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Real z = Ms[j][3 * c] * rs[j][0] + Ms[j][3 * c + 1] * rs[j][1] + Ms[j][3 * c + 2] * rs[j][2];
                zw[3 * (size_t)(lo + i) + c] = z;
                acc[0] += rs[j][c] * z;
                acc[1] += rs[j][c] * rs[j][c];
            }
        }
        if (own_a) {
            // q of the affine row component: the CTAs' partials in rank order
            // (independent remote loads first)
            Real qv[kPcgcMaxCluster];
#pragma unroll
            for (int rk = 0; rk < kPcgcMaxCluster; ++rk) qv[rk] = rk < cs ? cl.map_shared_rank(s_qa, rk)[tid] : Real(0);
            Real q = 0;
#pragma unroll
            for (int rk = 0; rk < kPcgcMaxCluster; ++rk) q += qv[rk];
            xa += alpha * s_p[PS * (ns1 - nb + tid / 3) + tid % 3];
            ra -= alpha * q;
            s_ra[tid] = ra;
        }
        __syncthreads();
        if (own_a) {
            const int bi = tid / 12;
            Real z = 0;
#pragma unroll
            for (int c = 0; c < 12; ++c) z += Ma[c] * s_ra[12 * bi + c];
            zw[3 * (size_t)ns1 + tid] = z;
            acc[0] += ra * z;
            acc[1] += ra * ra;
        }
        Real t2[2];
        cluster_allreduce<2>(cl, acc, s_red[1], s_w, t2);  // B2
        const Real rz_new = t2[0], rr = t2[1];
        ++it;
        if (!isfinite(rr)) bad = done = true;
        if (!(rr > stop2)) done = true;
        beta = rz != Real(0) ? rz_new / rz : Real(0);
        rz = rz_new;
    }
    it_total += it;
    // solution out (double) for the owned units: x of the first pass, plus
    // the correction d of each refinement round
#pragma unroll
    for (int j = 0; j < kPcgcOwn; ++j) {
        const int i = tid + j * kPcgcThreads;
        if (i >= n_own) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double* xo = a.x_out + 3 * (size_t)(lo + i) + c;
            *xo = pass ? *xo + (double)xs[j][c] : (double)xs[j][c];
        }
    }
    if (own_a) {
        double* xo = a.x_out + 3 * (size_t)ns1 + tid;
        *xo = pass ? *xo + (double)xa : (double)xa;
    }
    // 2: non-finite right-hand side or matrix; 3: max_iter reached first
    status = bad ? 2 : (done ? 1 : 3);
    if (status != 1 || pass >= a.refine) break;
    // ---- FP64 residual r = b - A x (FP64 products over the stored matrix),
    // |r|^2 and |b|^2; a correction solve of A d = r while |r|^2 > tol2 |b|^2
    cl.sync();  // x of every CTA written
    double acc64[2] = {0.0, 0.0};
    for (int tb = kGroupsPerWarp * warp; tb < n_tasks; tb += n_groups) {
        const int task = tb + sub;
        const bool valid = task < n_tasks;
        double y0 = 0.0, y1 = 0.0, y2 = 0.0;
        if (valid) {
            const int4 g = s_rng[task];
            row_part64(a, staged, s_mval, g, 0, (g.y - g.x) + (g.w - g.z), a.x_out, gl, y0, y1, y2);
        }
        y0 = group_sum(y0);
        y1 = group_sum(y1);
        y2 = group_sum(y2);
        if (valid && gl == 0) {
            if (task < n_own) {
                const size_t o = 3 * (size_t)(lo + task);
                const double b0 = a.b[o], b1 = a.b[o + 1], b2 = a.b[o + 2];
                const double r0 = b0 - y0, r1 = b1 - y1, r2 = b2 - y2;
                a.r64[o] = r0;
                a.r64[o + 1] = r1;
                a.r64[o + 2] = r2;
                acc64[0] += r0 * r0 + r1 * r1 + r2 * r2;
                acc64[1] += b0 * b0 + b1 * b1 + b2 * b2;
            } else {
                double* q = s_qa64 + 3 * (task - n_own);
                q[0] = y0;
                q[1] = y1;
                q[2] = y2;
            }
        }
    }
    cl.sync();  // the CTAs' partial products of the affine rows
    if (own_a) {
        double y = 0.0;
        for (int rk = 0; rk < cs; ++rk) y += cl.map_shared_rank(s_qa64, rk)[tid];
        const size_t o = 3 * (size_t)ns1 + tid;
        const double bv = a.b[o], r = bv - y;
        a.r64[o] = r;
        acc64[0] += r * r;
        acc64[1] += bv * bv;
    }
    double t64[2];
    cluster_allreduce<2>(cl, acc64, s_red64, s_w64, t64);
    if (!isfinite(t64[0])) {
        status = 2;
        break;
    }
    const double tol2 = a.tol2_env ? a.tol2_env[e] : a.tol2;
    if (!(t64[0] > tol2 * t64[1])) break;
    // the correction only has to bring |r - A d| under tol |b|: its solve
    // stops at half of that, relative to |r|
    ++n_ref;
    tol_pass = (Real)fmin(0.25, 0.25 * tol2 * t64[1] / t64[0]);
    init(a.r64, acc0);
    }
    if (rank == 0 && tid == 0) {
        a.iters[e] = it_total;
        a.conv[e] = status;
        if (a.refines) a.refines[e] = n_ref;
    }
    cl.sync();  // no CTA leaves while a partner may still read its shared memory
}

// The FP32 matrix packed for the cluster solve: block k of S, then block k
// of C at nS + k, as 12 floats (the 9 values, the column as int bits, 2 zero
// pads), so that an unstaged CTA reads a block with three 16-byte loads
// instead of ten scalar ones.  The C block count is read on the device; the
// blocks of converged envs are not written (their clusters return at once).
__global__ void k_pack_blocks(Geo G, Bsr<float> S, Bsr<float> C, int nS, const int* nC, float4* pk) {
    const long long n = (long long)nS + *nC;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const bool in_s = k < nS;
        const long long j = in_s ? k : k - nS;
        const int col = in_s ? S.col[j] : C.col[j];
        if (env_is_done(G, G.node_env[col])) continue;
        const float* v = (in_s ? S.val : C.val) + 9 * j;
        float4* o = pk + 3 * k;
        o[0] = make_float4(v[0], v[1], v[2], v[3]);
        o[1] = make_float4(v[4], v[5], v[6], v[7]);
        o[2] = make_float4(v[8], __int_as_float(col), 0.0f, 0.0f);
    }
}

// FP64 residual of an FP32 solve: r = b - A x per node (A the stored FP32
// matrix S + C, products and sums in FP64), zero for envs flagged in skip.
// One warp per row, lanes over the row's blocks, a fixed shuffle tree.
template <class T>
__global__ void k_residual64(Geo G, Bsr<T> S, Bsr<T> C, const double* x, const double* b, const int* skip,
                             double* r) {
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = (int)(gt >> 5), l = threadIdx.x & 31;
    if (n >= G.n_nodes) return;  // the whole warp
    if (skip[G.node_env[n]]) {  // the whole warp
        if (l < 3) r[3 * (size_t)n + l] = 0.0;
        return;
    }
    double y[3] = {0.0, 0.0, 0.0};
    for (int pass = 0; pass < 2; ++pass) {
        const Bsr<T>& A = pass ? C : S;
        for (int k = A.rowptr[n] + l; k < A.rowptr[n + 1]; k += 32) {
            const T* v = A.val + 9 * (size_t)k;
            const double* xc = x + 3 * (size_t)A.col[k];
            for (int i = 0; i < 3; ++i)
                y[i] += (double)v[3 * i] * xc[0] + (double)v[3 * i + 1] * xc[1] + (double)v[3 * i + 2] * xc[2];
        }
    }
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) y[i] += __shfl_xor_sync(0xffffffffu, y[i], o);
    if (l < 3) {
        const double yi = l == 0 ? y[0] : (l == 1 ? y[1] : y[2]);
        const size_t o = 3 * (size_t)n + l;
        r[o] = skip[G.node_env[n]] ? 0.0 : b[o] - yi;
    }
}

// p += dx on the envs flagged in need
__global__ void k_add_env(Geo G, double* p, const double* dx, const int* need) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.n_nodes || !need[G.node_env[n]]) return;
    for (int j = 0; j < 3; ++j) p[3 * (size_t)n + j] += dx[3 * (size_t)n + j];
}

}  // namespace zema
