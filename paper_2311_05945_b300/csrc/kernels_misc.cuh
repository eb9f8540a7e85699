// Predictor, surface positions, pair-list plumbing, additive CCD, step
// norms, velocity update and the kinematic augmented-Lagrangian bookkeeping.
#pragma once
#include "kernels_linear.cuh"

namespace zema {

// x^t <- x ; x^ = x^t + h v^t + h^2 g (soft nodes and affine p'), + h v (affine c_k)
// (Eq. 1-3; for affine bodies M_b^-1 f_e = (g, 0, 0, 0) in the centred form)
__global__ void k_predict(Geo G, const double* x, const double* v, double* xt, double* xhat, double gx, double gy,
                          double gz) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.n_nodes) return;
    V3 xn = ld3(x + 3 * (size_t)n);
    st3(xt + 3 * (size_t)n, xn);
    if (G.node_fixed[n]) {
        st3(xhat + 3 * (size_t)n, xn);
        return;
    }
    V3 vn = ld3(v + 3 * (size_t)n);
    double h = G.h;
    V3 r = xn + h * vn;
    // gravity on soft nodes here; on the p' node of affine bodies in k_predict_affine
    if (G.node_mass[n] > 0.0) r = r + (h * h) * v3(gx, gy, gz);
    st3(xhat + 3 * (size_t)n, r);
}

__global__ void k_predict_affine(Geo G, double* xhat, double gx, double gy, double gz) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= G.n_aff || G.aff_mode[b] == 1) return;
    double h2 = G.h * G.h;
    double* p = xhat + 3 * (size_t)G.aff_node0[b];
    p[0] += h2 * gx;
    p[1] += h2 * gy;
    p[2] += h2 * gz;
}

__global__ void k_sv_pos(Geo G, const double* x, double* X) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= G.n_sv) return;
    st3(X + 3 * (size_t)s, sv_pos(G, x, s));
}

// xo = x + alpha_env * p
__global__ void k_axpy_env(Geo G, const double* x, const double* p, const double* alpha, double* xo) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.n_nodes) return;
    double a = alpha[G.node_env[n]];
    for (int j = 0; j < 3; ++j) xo[3 * (size_t)n + j] = x[3 * (size_t)n + j] + a * p[3 * (size_t)n + j];
}

// zero the entries of environments that are flagged done
__global__ void k_mask_env(Geo G, double* p, const int* done) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.n_nodes) return;
    if (done[G.node_env[n]])
        for (int j = 0; j < 3; ++j) p[3 * (size_t)n + j] = 0.0;
}

__global__ void k_negate(const double* a, double* b, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = -a[i];
}

// max |component| of the step over soft nodes and over the displacement of
// affine surface vertices (J p_b), per env
__global__ void k_step_norm(Geo G, const double* p, double* part) {
    int env = blockIdx.y;
    __shared__ double sh[32];
    double m = 0.0;
    int n0 = G.env_node_start[env], n1 = G.env_node_start[env + 1];
    for (int n = n0 + blockIdx.x * blockDim.x + threadIdx.x; n < n1; n += gridDim.x * blockDim.x)
        if (G.node_mass[n] > 0.0) {
            V3 q = ld3(p + 3 * (size_t)n);
            m = fmax(m, fmax(fabs(q.x), fmax(fabs(q.y), fabs(q.z))));
        }
    int s0 = G.env_sv_start[env], s1 = G.env_sv_start[env + 1];
    for (int s = s0 + blockIdx.x * blockDim.x + threadIdx.x; s < s1; s += gridDim.x * blockDim.x)
        if (G.sv_aff[s]) {
            V3 q = sv_pos(G, p, s);
            m = fmax(m, fmax(fabs(q.x), fmax(fabs(q.y), fabs(q.z))));
        }
    double t = block_max(m, sh);
    if (threadIdx.x == 0) part[(size_t)env * kChunks + blockIdx.x] = t;
}

// ---------------------------------------------------------------------------
// Additive CCD (Li, Kaufman, Jiang 2021) with thickness 0: the common motion
// is removed, l_p bounds the closing speed, and the stencil advances by
// (1 - s) d / l_p, then 0.9 d / l_p, until d falls below s d_0.  Returns the
// safe fraction t in (0, t_c].
// ---------------------------------------------------------------------------
__device__ inline double accd(const V3* x0, const V3* p0, bool is_ee, double s, double tc, int max_iter,
                              int* hit_cap) {
    V3 x[4], p[4];
    V3 mean = 0.25 * (p0[0] + p0[1] + p0[2] + p0[3]);
    double nrm[4];
    for (int k = 0; k < 4; ++k) {
        x[k] = x0[k];
        p[k] = p0[k] - mean;
        nrm[k] = sqrt(dot(p[k], p[k]));
    }
    double lp = is_ee ? fmax(nrm[0], nrm[1]) + fmax(nrm[2], nrm[3]) : nrm[0] + fmax(nrm[1], fmax(nrm[2], nrm[3]));
    if (lp == 0.0) return tc;
    double d = sqrt(stencil_d2(x, is_ee));
    double gap = s * d;
    double t = 0.0;
    double tl = (1.0 - s) * d / lp;
    for (int it = 0; it < max_iter; ++it) {
        for (int k = 0; k < 4; ++k) x[k] = x[k] + tl * p[k];
        if (it == 0) {
            // t is 0 here, so the distance only sets the next advance: a
            // first advance past t_c (a pair far apart for its motion) ends
            // without it
            t += tl;
            if (t > tc) return tc;
            d = sqrt(stencil_d2(x, is_ee));
            tl = 0.9 * d / lp;
            continue;
        }
        d = sqrt(stencil_d2(x, is_ee));
        if (t > 0.0 && d < gap) return t;
        t += tl;
        if (t > tc) return tc;
        tl = 0.9 * d / lp;
    }
    if (hit_cap) *hit_cap = 1;
    return t;
}

__device__ __forceinline__ void load_stencil(const double* X, const PairRec& r, V3* x) {
    for (int k = 0; k < 4; ++k) x[k] = ld3(X + 3 * (size_t)r.s[k]);
}

// per-env min over pairs of the ACCD bound along X0 -> X1
__global__ void k_accd(Geo G, const double* X0, const double* X1, const PairRec* rec, int n, double* alpha_env,
                       int* cap_flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PairRec r = rec[i];
    V3 x[4], e[4], p[4];
    load_stencil(X0, r, x);
    load_stencil(X1, r, e);
    for (int k = 0; k < 4; ++k) p[k] = e[k] - x[k];
    int cap = 0;
    double t = accd(x, p, r.is_ee != 0, 0.1, 1.0, 10000, &cap);
    if (cap) *cap_flag = 1;
    atomic_min_pos(&alpha_env[G.sv_env[r.s[0]]], t);
}

// distance flags of candidates: active iff d < dhat; per-env minimum distance
__global__ void k_active_flags(Geo G, const double* X, const PairRec* rec, int n, uint32_t* flag, double* dmin_env) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PairRec r = rec[i];
    V3 x[4];
    load_stencil(X, r, x);
    if (stencil_beyond(x, r.is_ee != 0, G.dhat)) {
        flag[i] = 0u;
        return;
    }
    double d = sqrt(stencil_d2(x, r.is_ee != 0));
    bool a = d < G.dhat;
    flag[i] = a ? 1u : 0u;
    if (a && dmin_env) atomic_min_pos(&dmin_env[G.sv_env[r.s[0]]], d);
}

__global__ void k_compact_pairs(const PairRec* in, const uint32_t* flag, const uint32_t* off, int n, PairRec* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (flag[i]) out[off[i]] = in[i];
}

// per-env offsets of a compacted list: off_out[e] = scan[start[e]]
__global__ void k_env_gather(const uint32_t* scan, const uint32_t* start, int n_envs, uint32_t* out) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e > n_envs) return;
    out[e] = scan[start[e]];
}

// env offsets of the PT (by surface vertex) and EE (by edge) candidate lists
// and of their per-env merge
// per env, the first PT pair, EE pair and merged pair of its queries; the
// broad phase covered the local point queries [sv_base, sv_base + nsv) and
// edge queries [edge_base, edge_base + ne) (qoff_* over those, n + 1 each)
__global__ void k_pair_env_offsets(Geo G, const uint32_t* qoff_pt, const uint32_t* qoff_ee, int sv_base, int nsv,
                                   int edge_base, int ne, uint32_t* pt_env, uint32_t* ee_env, uint32_t* m_env) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e > G.n_envs) return;
    const int ip = min(max(G.env_sv_start[e] - sv_base, 0), nsv), ie = min(max(G.env_edge_start[e] - edge_base, 0), ne);
    uint32_t a = qoff_pt[ip], b = qoff_ee[ie];
    pt_env[e] = a;
    ee_env[e] = b;
    m_env[e] = a + b;
}

// merged, env-ordered pair records: per env its PT pairs then its EE pairs
__global__ void k_merge_pairs(Geo G, const int2* pt, const int2* ee, const uint32_t* pt_env, const uint32_t* ee_env,
                              const uint32_t* m_env, int n, PairRec* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = G.n_envs - 1;
    while (lo < hi) {  // last env with m_env[e] <= i
        int mid = (lo + hi + 1) >> 1;
        if (m_env[mid] <= (uint32_t)i)
            lo = mid;
        else
            hi = mid - 1;
    }
    int e = lo;
    uint32_t j = (uint32_t)i - m_env[e];
    uint32_t npt = pt_env[e + 1] - pt_env[e];
    PairRec r;
    if (j < npt) {
        int2 q = pt[pt_env[e] + j];
        int3 t = G.tris[q.y];
        r.s[0] = q.x;
        r.s[1] = t.x;
        r.s[2] = t.y;
        r.s[3] = t.z;
        r.is_ee = 0;
    } else {
        int2 q = ee[ee_env[e] + (j - npt)];
        int2 a = G.edges[q.x], b = G.edges[q.y];
        r.s[0] = a.x;
        r.s[1] = a.y;
        r.s[2] = b.x;
        r.s[3] = b.y;
        r.is_ee = 1;
    }
    out[i] = r;
}

// v = (x - x^t) / h (Eq. 11)
__global__ void k_velocity(Geo G, const double* x, const double* xt, double* v) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.n_nodes) return;
    double ih = 1.0 / G.h;
    for (int j = 0; j < 3; ++j) {
        size_t o = 3 * (size_t)n + j;
        v[o] = G.node_fixed[n] ? 0.0 : (x[o] - xt[o]) * ih;
    }
}

// E[env] = sum over terms and chunks of the partials (fixed order)
__global__ void k_energy_total(const double* part, int n_terms, int n_envs, double* E) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_envs) return;
    double s = 0.0;
    for (int t = 0; t < n_terms; ++t)
        for (int c = 0; c < kChunks; ++c) s += part[((size_t)t * n_envs + e) * kChunks + c];
    E[e] = s;
}

__global__ void k_max_total(const double* part, int n_envs, double* out) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_envs) return;
    double s = 0.0;
    for (int c = 0; c < kChunks; ++c) s = fmax(s, part[(size_t)e * kChunks + c]);
    out[e] = s;
}

// dot products per env of two node vectors (partials), for the kappa rule
__global__ void k_env_dot2(Geo G, const double* a, const double* b, double* part_ab, double* part_bb) {
    int env = blockIdx.y;
    __shared__ double sh[32];
    double sab = 0.0, sbb = 0.0;
    int n0 = G.env_node_start[env], n1 = G.env_node_start[env + 1];
    for (int n = n0 + blockIdx.x * blockDim.x + threadIdx.x; n < n1; n += gridDim.x * blockDim.x) {
        V3 x = ld3(a + 3 * (size_t)n), y = ld3(b + 3 * (size_t)n);
        sab += dot(x, y);
        sbb += dot(y, y);
    }
    double t1 = block_sum<kRedThreads>(sab, sh);
    double t2 = block_sum<kRedThreads>(sbb, sh);
    if (threadIdx.x == 0) {
        part_ab[(size_t)env * kChunks + blockIdx.x] = t1;
        part_bb[(size_t)env * kChunks + blockIdx.x] = t2;
    }
}

// Gradient of the affine nodes converted to the caller's row form in place
// (the paper's DOF coordinates), used where dot products of gradients need
// those coordinates: g_row = L^T g_col with p' = p + A com, c_k = A e_k.
__global__ void k_affine_grad_to_row(Geo G, double* g) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= G.n_aff) return;
    double* q = g + 3 * (size_t)G.aff_node0[b];
    const double* com = G.aff_com + 3 * (size_t)b;
    double gp[3] = {q[0], q[1], q[2]};
    double gc[3][3];
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i) gc[k][i] = q[3 + 3 * k + i];
    // dE/dp = dE/dp' ; dE/dA_ik = dE/dc_k[i] + dE/dp'_i com_k
    double out[12];
    for (int i = 0; i < 3; ++i) out[i] = gp[i];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) out[3 + 3 * i + k] = gc[k][i] + gp[i] * com[k];
    for (int j = 0; j < 12; ++j) q[j] = out[j];
}

// kinematic AL: largest |q - q~| (row form) per env, and the multiplier update
__device__ __forceinline__ void aff_row_q(const Geo& G, const double* x, int b, double* q) {
    int n0 = G.aff_node0[b];
    V3 c[4];
    for (int j = 0; j < 4; ++j) c[j] = ld3(x + 3 * (size_t)(n0 + j));
    const double* com = G.aff_com + 3 * (size_t)b;
    V3 p = c[0] - (com[0] * c[1] + com[1] * c[2] + com[2] * c[3]);
    q[0] = p.x;
    q[1] = p.y;
    q[2] = p.z;
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) q[3 + 3 * i + k] = comp(c[1 + k], i);
}

__global__ void k_al_check(Geo G, const double* x, AffKin K, const double* tol_env, int* need_env) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= G.n_aff || G.aff_mode[b] != 2) return;
    double q[12];
    aff_row_q(G, x, b, q);
    double m = 0.0;
    for (int i = 0; i < 12; ++i) m = fmax(m, fabs(q[i] - K.qtarget[12 * (size_t)b + i]));
    int env = G.node_env[G.aff_node0[b]];
    if (m > tol_env[env]) atomicMax(&need_env[env], 1);
}

// lambda_A -= kappa_A (q - q~) / sqrt(m) for the kinematic bodies of the envs
// flagged in need_env (all envs when need_env is NULL)
__global__ void k_al_update(Geo G, const double* x, const double* qtarget, double* lamA, const int* need_env) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= G.n_aff || G.aff_mode[b] != 2) return;
    int env = G.node_env[G.aff_node0[b]];
    if (need_env && !need_env[env]) return;
    double q[12];
    aff_row_q(G, x, b, q);
    double m = G.aff_m[b];
    double kA = 1e3 * m, sm = sqrt(m);
    for (int i = 0; i < 12; ++i) lamA[12 * (size_t)b + i] -= kA * (q[i] - qtarget[12 * (size_t)b + i]) / sm;
}

}  // namespace zema
