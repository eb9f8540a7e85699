// Learned Newton warm start: per-soft-vertex features at x^t, and the
// proposal direction from the network's output.
//
// Features of soft vertex i of body b (13 values, FP32):
//   (x_i - c_b) / R_b          position relative to the body's centroid c_b,
//                              over the body's rest half-diagonal R_b
//   v_i h / s                  constant-velocity displacement
//   (xhat_i - x_i) / s         displacement to the inertial target (Eq. 1)
//   min(d_i / dhat, 1)         distance of the nearest active pair at x^t
//   n_i                        its unit normal, pointing away from the other
//                              primitive (0 when no pair is active)
// with s = h^2 |g| the free-fall displacement of one step.  The network
// predicts the step's displacement beyond the constant-velocity one,
// y = (x^{t+1} - x^t - h v^t) / s.  The step applies the constant-velocity
// proposal first and then the correction s y from there, each CCD-bounded and
// kept only if the energy does not rise, so the learned start is never worse
// in energy than the constant-velocity one; Newton then runs to the same
// tolerance.
//
// Features of dynamic affine body b (40 values, FP32), for the per-body
// network; q = (p, c1, c2, c3) with the c_k the columns of A:
//   c1, c2, c3                 orientation (9)
//   (p - c_env) / D_env        position relative to the env's rest bounding
//                              box centre, over its diagonal (3)
//   h qdot / s                 constant-velocity displacement (12)
//   (qhat - q) / s             displacement to the inertial target (12)
//   min(d / dhat, 1), n        nearest active pair touching the body and its
//                              normal pointing away from the other primitive (4)
// where the A parts are multiplied by the body's rest half-diagonal R_b, so
// that every displacement is in metres of surface motion before the scaling
// by s.  The network predicts the step's change of q beyond h qdot in the
// same units (12 outputs).
#pragma once
#include "kernels_energy.cuh"

namespace zema {

constexpr int kWsFeatures = 13;
constexpr int kWsOutputs = 3;
constexpr int kWsAffFeatures = 40;
constexpr int kWsAffOutputs = 12;
constexpr int kWsHalvings = 0;  // halvings of the learned correction (a single energy check)

// sign of a pair's normal seen from node n (+1: the normal points away from
// the other primitive), 0 when the node takes no part with nonzero weight
__device__ __forceinline__ float ws_side(const Geo& G, const PairRec& r, const double* w4, int n, bool aff) {
    float sg = 0.0f;
    for (int k = 0; k < 4; ++k)
        if ((G.sv_aff[r.s[k]] != 0) == aff && G.sv_node[r.s[k]] == n && w4[k] != 0.0) sg = w4[k] > 0.0 ? 1.0f : -1.0f;
    return sg;
}

// centroid of each tet body at x: one block per body, fixed-order sums
__global__ void k_ws_centroid(const double* x, const int* node0, const int* nv, double* c) {
    __shared__ double sh[32];
    const int b = blockIdx.x, n0 = node0[b], m = nv[b];
    double s[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        for (int j = 0; j < 3; ++j) s[j] += x[3 * (size_t)(n0 + i) + j];
    for (int j = 0; j < 3; ++j) {
        double t = block_sum<kRedThreads>(s[j], sh);
        if (threadIdx.x == 0) c[3 * b + j] = m ? t / m : 0.0;
    }
}

// nearest active pair of every soft vertex: 64-bit key (distance bits, pair
// index); atomicMin of such keys gives the same winner in any order
__global__ void k_ws_nearest(Geo G, const double* X, const PairRec* rec, const double* w, int n,
                             unsigned long long* best) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const PairRec r = rec[i];
    V3 dv = v3(0, 0, 0);
    for (int k = 0; k < 4; ++k) dv = dv + w[4 * (size_t)i + k] * ld3(X + 3 * (size_t)r.s[k]);
    const float d = (float)sqrt(dot(dv, dv));
    const unsigned long long key = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)i;
    for (int k = 0; k < 4; ++k) {
        const int sv = r.s[k];
        if (w[4 * (size_t)i + k] == 0.0) continue;
        atomicMin(best + G.sv_node[sv], key);  // soft: its node; affine: the body's first node
    }
}

__global__ void k_ws_features(Geo G, const int* soft, const int* sbody, int ns, const double* x, const double* v,
                              const double* xhat, const double* cen, const double* R,
                              const unsigned long long* best, const PairRec* rec, const double* w,
                              const double* nrm, double h, double sc, float* f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const int n = soft[i], b = sbody[i];
    float* o = f + (size_t)kWsFeatures * i;
    const double iR = 1.0 / R[b], is = 1.0 / sc;
    for (int j = 0; j < 3; ++j) {
        const double xj = x[3 * (size_t)n + j];
        o[j] = (float)((xj - cen[3 * b + j]) * iR);
        o[3 + j] = (float)(v[3 * (size_t)n + j] * h * is);
        o[6 + j] = (float)((xhat[3 * (size_t)n + j] - xj) * is);
    }
    const unsigned long long key = best[n];
    float dn = 1.0f, nv[3] = {0.0f, 0.0f, 0.0f};
    if (key != ~0ull) {
        const unsigned p = (unsigned)(key & 0xffffffffull);
        dn = fminf(__uint_as_float((unsigned)(key >> 32)) / (float)G.dhat, 1.0f);
        const float sg = ws_side(G, rec[p], w + 4 * (size_t)p, n, false);
        for (int j = 0; j < 3; ++j) nv[j] = sg * (float)nrm[3 * (size_t)p + j];
    }
    o[9] = dn;
    o[10] = nv[0];
    o[11] = nv[1];
    o[12] = nv[2];
}

__global__ void k_ws_aff_features(Geo G, const int* aff, int na, const double* x, const double* v, const double* xhat,
                                  const double* Rb, const double* env_c, const double* env_d,
                                  const unsigned long long* best, const PairRec* rec, const double* w,
                                  const double* nrm, double h, double sc, float* f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= na) return;
    const int a = aff[i], n0 = G.aff_node0[a], e = G.node_env[n0];
    float* o = f + (size_t)kWsAffFeatures * i;
    const double is = 1.0 / sc, R = Rb[i];
    for (int k = 1; k < 4; ++k)
        for (int j = 0; j < 3; ++j) o[3 * (k - 1) + j] = (float)x[3 * (size_t)(n0 + k) + j];
    for (int j = 0; j < 3; ++j) o[9 + j] = (float)((x[3 * (size_t)n0 + j] - env_c[3 * e + j]) / env_d[e]);
    for (int k = 0; k < 4; ++k) {
        const double m = k == 0 ? is : R * is;
        for (int j = 0; j < 3; ++j) {
            const size_t q = 3 * (size_t)(n0 + k) + j;
            o[12 + 3 * k + j] = (float)(v[q] * h * m);
            o[24 + 3 * k + j] = (float)((xhat[q] - x[q]) * m);
        }
    }
    const unsigned long long key = best[n0];
    float dn = 1.0f, nv[3] = {0.0f, 0.0f, 0.0f};
    if (key != ~0ull) {
        const unsigned p = (unsigned)(key & 0xffffffffull);
        dn = fminf(__uint_as_float((unsigned)(key >> 32)) / (float)G.dhat, 1.0f);
        const float sg = ws_side(G, rec[p], w + 4 * (size_t)p, n0, true);
        for (int j = 0; j < 3; ++j) nv[j] = sg * (float)nrm[3 * (size_t)p + j];
    }
    o[36] = dn;
    o[37] = nv[0];
    o[38] = nv[1];
    o[39] = nv[2];
}

// correction direction of the dynamic affine bodies: dir(q) += s y, the A
// part divided by R_b
__global__ void k_ws_aff_direction(Geo G, const int* aff, int na, const double* Rb, const float* out, double sc,
                                   double* dir) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= na) return;
    const int n0 = G.aff_node0[aff[i]];
    for (int k = 0; k < 4; ++k) {
        const double m = k == 0 ? sc : sc / Rb[i];
        for (int j = 0; j < 3; ++j)
            dir[3 * (size_t)(n0 + k) + j] += m * (double)out[(size_t)kWsAffOutputs * i + 3 * k + j];
    }
}

// training target of the per-body network: the change of q beyond h qdot^t
// in the feature units (features 12..23 hold h qdot^t in those units)
__global__ void k_ws_aff_target(Geo G, const int* aff, int na, const double* Rb, const double* x1, const double* x0,
                                const float* feat, double sc, float* t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= na) return;
    const int n0 = G.aff_node0[aff[i]];
    for (int k = 0; k < 4; ++k) {
        const double m = k == 0 ? 1.0 / sc : Rb[i] / sc;
        for (int j = 0; j < 3; ++j) {
            const size_t q = 3 * (size_t)(n0 + k) + j;
            t[(size_t)kWsAffOutputs * i + 3 * k + j] =
                (float)((x1[q] - x0[q]) * m - (double)feat[(size_t)kWsAffFeatures * i + 12 + 3 * k + j]);
        }
    }
}

// correction direction of the soft vertices: dir += s y
__global__ void k_ws_direction(const int* soft, int ns, const float* out, double sc, double* dir) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const int n = soft[i];
    for (int j = 0; j < 3; ++j) dir[3 * (size_t)n + j] += sc * (double)out[(size_t)kWsOutputs * i + j];
}

// training target: the step's displacement beyond h v^t, over s (features
// 3..5 hold h v^t / s)
__global__ void k_ws_target(const int* soft, int ns, const double* x1, const double* x0, const float* feat,
                            double sc, float* t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const int n = soft[i];
    for (int j = 0; j < 3; ++j)
        t[(size_t)kWsOutputs * i + j] = (float)((x1[3 * (size_t)n + j] - x0[3 * (size_t)n + j]) / sc -
                                                (double)feat[(size_t)kWsFeatures * i + 3 + j]);
}

}  // namespace zema
