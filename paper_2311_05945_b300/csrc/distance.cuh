// Point-triangle / edge-edge distances for the contact barrier (Eq. 5, Eq. 6-8).
//
// A pair is a 4-point stencil: PT = (p, t0, t1, t2), EE = (a0, a1, b0, b1).
// The closest features are classified by region tests; d^2 is then written as
// a function of 1-3 difference vectors ("reduced variables") whose derivatives
// have closed forms, and mapped back to the 12 stencil coordinates by a
// constant coefficient matrix.
#pragma once
#include "common.cuh"

namespace zema {

enum DistType : int { DT_PP = 0, DT_PE = 1, DT_PT = 2, DT_EE = 3 };

struct DistInfo {
    double d2;
    int type;
    int s[3];     // PP: (i, j); PE: (p, e0, e1) stencil slots
    double w[4];  // closest-point weights: Delta = sum_k w[k] x_k
};

// squared distance from point p to segment [a, b]; t in [0, 1] the clamped parameter
__device__ __forceinline__ double seg_d2(V3 p, V3 a, V3 b, double& t) {
    V3 e = b - a;
    double ee = dot(e, e);
    t = ee > 0.0 ? dot(p - a, e) / ee : 0.0;
    t = fmin(fmax(t, 0.0), 1.0);
    V3 c = p - (a + t * e);
    return dot(c, c);
}

// point slot i against segment slots (j, k): fills info if closer
__device__ __forceinline__ void pe_candidate(const V3* x, int i, int j, int k, double sgn, DistInfo& di) {
    double t;
    double d2 = seg_d2(x[i], x[j], x[k], t);
    if (!(d2 < di.d2)) return;
    di.d2 = d2;
    for (int m = 0; m < 4; ++m) di.w[m] = 0.0;
    if (t <= 0.0) {
        di.type = DT_PP;
        di.s[0] = i;
        di.s[1] = j;
        di.w[i] = sgn;
        di.w[j] = -sgn;
    } else if (t >= 1.0) {
        di.type = DT_PP;
        di.s[0] = i;
        di.s[1] = k;
        di.w[i] = sgn;
        di.w[k] = -sgn;
    } else {
        di.type = DT_PE;
        di.s[0] = i;
        di.s[1] = j;
        di.s[2] = k;
        di.w[i] = sgn;
        di.w[j] = -sgn * (1.0 - t);
        di.w[k] = -sgn * t;
    }
}

// Point-triangle: interior when the point projects inside all three edges,
// else the nearest point on the triangle boundary.
__device__ inline DistInfo classify_pt(const V3* x) {
    DistInfo di;
    di.d2 = 1e300;
    di.type = DT_PP;
    V3 p = x[0], t0 = x[1], t1 = x[2], t2 = x[3];
    V3 n = cross(t1 - t0, t2 - t0);
    double nn = dot(n, n);
    if (nn > 0.0) {
        double s0 = dot(cross(t1 - t0, p - t0), n);
        double s1 = dot(cross(t2 - t1, p - t1), n);
        double s2 = dot(cross(t0 - t2, p - t2), n);
        if (s0 >= 0.0 && s1 >= 0.0 && s2 >= 0.0) {
            double h = dot(p - t0, n);
            di.d2 = h * h / nn;
            di.type = DT_PT;
            di.w[0] = 1.0;
            di.w[1] = -s1 / nn;  // barycentric weight of t0 (area opposite t0)
            di.w[2] = -s2 / nn;
            di.w[3] = -s0 / nn;
            return di;
        }
    }
    pe_candidate(x, 0, 1, 2, 1.0, di);
    pe_candidate(x, 0, 2, 3, 1.0, di);
    pe_candidate(x, 0, 3, 1, 1.0, di);
    return di;
}

// Edge-edge: interior-interior for non-parallel edges whose line parameters
// are both inside (0, 1), else the nearest endpoint-segment pair.
__device__ inline DistInfo classify_ee(const V3* x) {
    DistInfo di;
    di.d2 = 1e300;
    di.type = DT_PP;
    V3 ea = x[1] - x[0], eb = x[3] - x[2], r = x[0] - x[2];
    double A = dot(ea, ea), B = dot(ea, eb), C = dot(eb, eb), D = dot(ea, r), E = dot(eb, r);
    V3 cr = cross(ea, eb);
    double crn = dot(cr, cr);
    if (crn > 1e-20 * A * C) {
        double den = A * C - B * B;
        double s = (B * E - C * D) / den;
        double t = (A * E - B * D) / den;
        if (s > 0.0 && s < 1.0 && t > 0.0 && t < 1.0) {
            double h = dot(r, cr);
            di.d2 = h * h / crn;
            di.type = DT_EE;
            di.w[0] = 1.0 - s;
            di.w[1] = s;
            di.w[2] = -(1.0 - t);
            di.w[3] = -t;
            return di;
        }
    }
    pe_candidate(x, 0, 2, 3, 1.0, di);
    pe_candidate(x, 1, 2, 3, 1.0, di);
    pe_candidate(x, 2, 0, 1, -1.0, di);
    pe_candidate(x, 3, 0, 1, -1.0, di);
    return di;
}

__device__ __forceinline__ DistInfo classify(const V3* x, bool is_ee) {
    return is_ee ? classify_ee(x) : classify_pt(x);
}

__device__ __forceinline__ double stencil_d2(const V3* x, bool is_ee) { return classify(x, is_ee).d2; }

// ---------------------------------------------------------------------------
// Derivatives in the reduced variables.  A reduced variable k is
// sum_slot C[k][slot] x_slot with C entries in {-1, 0, 1}.
// ---------------------------------------------------------------------------
struct Red {
    int m;           // number of reduced 3-vectors (1..3)
    int C[3][4];     // coefficients
};

// Scatter a reduced 3x3 block (k, l) into the 12x12 slot-space matrix H.
__device__ __forceinline__ void scatter_block(SMat<12> H, const Red& R, int k, int l, const double* M, double sc) {
    for (int i = 0; i < 4; ++i) {
        int ci = R.C[k][i];
        if (!ci) continue;
        for (int j = 0; j < 4; ++j) {
            int cj = R.C[l][j];
            if (!cj) continue;
            double f = sc * ci * cj;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) H(3 * i + a, 3 * j + b) += f * M[3 * a + b];
        }
    }
}

__device__ __forceinline__ void scatter_grad(double* g12, const Red& R, int k, V3 v, double sc) {
    for (int i = 0; i < 4; ++i) {
        int ci = R.C[k][i];
        if (!ci) continue;
        g12[3 * i] += sc * ci * v.x;
        g12[3 * i + 1] += sc * ci * v.y;
        g12[3 * i + 2] += sc * ci * v.z;
    }
}

__device__ __forceinline__ void outer(double* M, V3 a, V3 b, double s) {
    double av[3] = {a.x, a.y, a.z}, bv[3] = {b.x, b.y, b.z};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] += s * av[i] * bv[j];
}
__device__ __forceinline__ void add_diag(double* M, double s) {
    M[0] += s;
    M[4] += s;
    M[8] += s;
}
__device__ __forceinline__ void add_skew(double* M, V3 v, double s) {  // M += s [v]x
    M[1] += -s * v.z;
    M[2] += s * v.y;
    M[3] += s * v.z;
    M[5] += -s * v.x;
    M[6] += -s * v.y;
    M[7] += s * v.x;
}
__device__ __forceinline__ void zero9(double* M) {
    for (int i = 0; i < 9; ++i) M[i] = 0.0;
}
__device__ __forceinline__ void transpose9(const double* M, double* T) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[3 * j + i] = M[3 * i + j];
}

// N = |a x b|^2: gradient (Na, Nb) and Hessian blocks (Haa, Hbb, Hab)
__device__ __forceinline__ void cross_norm_derivs(V3 a, V3 b, V3& Na, V3& Nb, double* Haa, double* Hbb,
                                                  double* Hab) {
    double aa = dot(a, a), bb = dot(b, b), ab = dot(a, b);
    Na = 2.0 * (bb * a - ab * b);
    Nb = 2.0 * (aa * b - ab * a);
    if (Haa) {
        zero9(Haa);
        add_diag(Haa, 2.0 * bb);
        outer(Haa, b, b, -2.0);
        zero9(Hbb);
        add_diag(Hbb, 2.0 * aa);
        outer(Hbb, a, a, -2.0);
        zero9(Hab);
        outer(Hab, a, b, 4.0);
        outer(Hab, b, a, -2.0);
        add_diag(Hab, -2.0 * ab);
    }
}

// f = d^2 of the classified type: value, slot gradient g12 and (when H.b is
// not null) slot Hessian accumulated into H (which must be zero on entry).
__device__ inline double d2_derivs(const V3* x, bool is_ee, const DistInfo& di, double* g12, SMat<12> H,
                                   bool want_h) {
    for (int i = 0; i < 12; ++i) g12[i] = 0.0;
    Red R;
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 4; ++i) R.C[k][i] = 0;
    if (di.type == DT_PP) {
        R.m = 1;
        R.C[0][di.s[0]] = 1;
        R.C[0][di.s[1]] = -1;
        V3 r = x[di.s[0]] - x[di.s[1]];
        scatter_grad(g12, R, 0, r, 2.0);
        if (want_h) {
            double M[9];
            zero9(M);
            add_diag(M, 2.0);
            scatter_block(H, R, 0, 0, M, 1.0);
        }
        return dot(r, r);
    }
    if (di.type == DT_PE) {
        R.m = 2;
        R.C[0][di.s[0]] = 1;
        R.C[0][di.s[1]] = -1;  // r = p - e0
        R.C[1][di.s[2]] = 1;
        R.C[1][di.s[1]] = -1;  // e = e1 - e0
        V3 r = x[di.s[0]] - x[di.s[1]];
        V3 e = x[di.s[2]] - x[di.s[1]];
        double L = dot(e, e), s = dot(r, e);
        double f = dot(r, r) - s * s / L;
        scatter_grad(g12, R, 0, 2.0 * r - (2.0 * s / L) * e, 1.0);
        scatter_grad(g12, R, 1, (-2.0 * s / L) * r + (2.0 * s * s / (L * L)) * e, 1.0);
        if (want_h) {
            double Hrr[9], Hre[9], Her[9], Hee[9];
            zero9(Hrr);
            add_diag(Hrr, 2.0);
            outer(Hrr, e, e, -2.0 / L);
            zero9(Hre);
            outer(Hre, e, r, -2.0 / L);
            add_diag(Hre, -2.0 * s / L);
            outer(Hre, e, e, 4.0 * s / (L * L));
            transpose9(Hre, Her);
            zero9(Hee);
            outer(Hee, r, r, -2.0 / L);
            outer(Hee, r, e, 4.0 * s / (L * L));
            outer(Hee, e, r, 4.0 * s / (L * L));
            add_diag(Hee, 2.0 * s * s / (L * L));
            outer(Hee, e, e, -8.0 * s * s / (L * L * L));
            scatter_block(H, R, 0, 0, Hrr, 1.0);
            scatter_block(H, R, 0, 1, Hre, 1.0);
            scatter_block(H, R, 1, 0, Her, 1.0);
            scatter_block(H, R, 1, 1, Hee, 1.0);
        }
        return f;
    }
    // plane (PT) or line-line (EE): f = (r . (a x b))^2 / |a x b|^2
    R.m = 3;
    if (!is_ee) {  // r = p - t0, a = t1 - t0, b = t2 - t0
        R.C[0][0] = 1;
        R.C[0][1] = -1;
        R.C[1][2] = 1;
        R.C[1][1] = -1;
        R.C[2][3] = 1;
        R.C[2][1] = -1;
    } else {  // r = a0 - b0, a = a1 - a0, b = b1 - b0
        R.C[0][0] = 1;
        R.C[0][2] = -1;
        R.C[1][1] = 1;
        R.C[1][0] = -1;
        R.C[2][3] = 1;
        R.C[2][2] = -1;
    }
    V3 r, a, b;
    if (!is_ee) {
        r = x[0] - x[1];
        a = x[2] - x[1];
        b = x[3] - x[1];
    } else {
        r = x[0] - x[2];
        a = x[1] - x[0];
        b = x[3] - x[2];
    }
    V3 n = cross(a, b);
    double N = dot(n, n), s = dot(r, n);
    double f = s * s / N;
    V3 sr = n, sa = cross(b, r), sb = cross(r, a);
    V3 Na, Nb;
    double Haa[9], Hbb[9], Hab[9];
    cross_norm_derivs(a, b, Na, Nb, want_h ? Haa : nullptr, Hbb, Hab);
    double c1 = 2.0 * s / N, c2 = -s * s / (N * N);
    scatter_grad(g12, R, 0, sr, c1);
    scatter_grad(g12, R, 1, c1 * sa + c2 * Na, 1.0);
    scatter_grad(g12, R, 2, c1 * sb + c2 * Nb, 1.0);
    if (want_h) {
        // grad s and grad N per reduced variable
        V3 S[3] = {sr, sa, sb};
        V3 Ng[3] = {v3(0, 0, 0), Na, Nb};
        const double iN = 1.0 / N, iN2 = iN * iN, iN3 = iN2 * iN;
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) {
                double M[9];
                zero9(M);
                outer(M, S[k], S[l], 2.0 * iN);
                outer(M, S[k], Ng[l], -2.0 * s * iN2);
                outer(M, Ng[k], S[l], -2.0 * s * iN2);
                outer(M, Ng[k], Ng[l], 2.0 * s * s * iN3);
                // (2 s / N) d2s/dk dl : trilinear s = r . (a x b)
                double cs = 2.0 * s * iN;
                if (k == 0 && l == 1) add_skew(M, b, -cs);  // dn/da = -[b]x
                if (k == 1 && l == 0) add_skew(M, b, cs);   // transpose of -[b]x
                if (k == 0 && l == 2) add_skew(M, a, cs);   // dn/db = [a]x
                if (k == 2 && l == 0) add_skew(M, a, -cs);
                if (k == 1 && l == 2) add_skew(M, r, -cs);  // d(b x r)/db = -[r]x
                if (k == 2 && l == 1) add_skew(M, r, cs);
                // -(s^2 / N^2) d2N
                double cn = -s * s * iN2;
                if (k == 1 && l == 1)
                    for (int q = 0; q < 9; ++q) M[q] += cn * Haa[q];
                if (k == 2 && l == 2)
                    for (int q = 0; q < 9; ++q) M[q] += cn * Hbb[q];
                if (k == 1 && l == 2)
                    for (int q = 0; q < 9; ++q) M[q] += cn * Hab[q];
                if (k == 2 && l == 1) {
                    double T[9];
                    transpose9(Hab, T);
                    for (int q = 0; q < 9; ++q) M[q] += cn * T[q];
                }
                scatter_block(H, R, k, l, M, 1.0);
            }
    }
    return f;
}

// ---------------------------------------------------------------------------
// Hessian of f = d^2 in the arithmetic type T (float in the mixed-precision
// mode).  The reduced vectors (differences of the stencil's points) are
// formed in FP64 and then rounded to T, so no cancellation happens in T; the
// formulas are those of d2_derivs above.
// ---------------------------------------------------------------------------
template <class T>
struct V3t {
    T x, y, z;
};
template <class T>
__device__ __forceinline__ V3t<T> to_t(V3 v) {
    return V3t<T>{(T)v.x, (T)v.y, (T)v.z};
}
template <class T>
__device__ __forceinline__ T dot_t(V3t<T> a, V3t<T> b) {
    return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <class T>
__device__ __forceinline__ V3t<T> cross_t(V3t<T> a, V3t<T> b) {
    return V3t<T>{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T>
__device__ __forceinline__ void outer_t(T* M, V3t<T> a, V3t<T> b, T s) {
    T av[3] = {a.x, a.y, a.z}, bv[3] = {b.x, b.y, b.z};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] += s * av[i] * bv[j];
}
template <class T>
__device__ __forceinline__ void add_diag_t(T* M, T s) {
    M[0] += s;
    M[4] += s;
    M[8] += s;
}
template <class T>
__device__ __forceinline__ void add_skew_t(T* M, V3t<T> v, T s) {  // M += s [v]x
    M[1] += -s * v.z;
    M[2] += s * v.y;
    M[3] += s * v.z;
    M[5] += -s * v.x;
    M[6] += -s * v.y;
    M[7] += s * v.x;
}
template <class T>
__device__ __forceinline__ void zero9_t(T* M) {
#pragma unroll
    for (int i = 0; i < 9; ++i) M[i] = T(0);
}
template <class T>
__device__ __forceinline__ void scatter_block_t(SMat<12, T> H, const Red& R, int k, int l, const T* M, T sc) {
    for (int i = 0; i < 4; ++i) {
        int ci = R.C[k][i];
        if (!ci) continue;
        for (int j = 0; j < 4; ++j) {
            int cj = R.C[l][j];
            if (!cj) continue;
            T f = sc * (T)(ci * cj);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) H(3 * i + a, 3 * j + b) += f * M[3 * a + b];
        }
    }
}
// Hessian blocks of N = |a x b|^2
template <class T>
__device__ __forceinline__ void cross_norm_hess_t(V3t<T> a, V3t<T> b, T* Haa, T* Hbb, T* Hab) {
    T aa = dot_t(a, a), bb = dot_t(b, b), ab = dot_t(a, b);
    zero9_t(Haa);
    add_diag_t(Haa, T(2) * bb);
    outer_t(Haa, b, b, T(-2));
    zero9_t(Hbb);
    add_diag_t(Hbb, T(2) * aa);
    outer_t(Hbb, a, a, T(-2));
    zero9_t(Hab);
    outer_t(Hab, a, b, T(4));
    outer_t(Hab, b, a, T(-2));
    add_diag_t(Hab, T(-2) * ab);
}

// reduced variables of the classified type (coefficients in R)
__device__ __forceinline__ void reduced_vars(const V3* x, bool is_ee, const DistInfo& di, Red& R, V3* v) {
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 4; ++i) R.C[k][i] = 0;
    if (di.type == DT_PP) {
        R.m = 1;
        R.C[0][di.s[0]] = 1;
        R.C[0][di.s[1]] = -1;
        v[0] = x[di.s[0]] - x[di.s[1]];
    } else if (di.type == DT_PE) {
        R.m = 2;
        R.C[0][di.s[0]] = 1;
        R.C[0][di.s[1]] = -1;
        R.C[1][di.s[2]] = 1;
        R.C[1][di.s[1]] = -1;
        v[0] = x[di.s[0]] - x[di.s[1]];
        v[1] = x[di.s[2]] - x[di.s[1]];
    } else if (!is_ee) {
        R.m = 3;
        R.C[0][0] = 1;
        R.C[0][1] = -1;
        R.C[1][2] = 1;
        R.C[1][1] = -1;
        R.C[2][3] = 1;
        R.C[2][1] = -1;
        v[0] = x[0] - x[1];
        v[1] = x[2] - x[1];
        v[2] = x[3] - x[1];
    } else {
        R.m = 3;
        R.C[0][0] = 1;
        R.C[0][2] = -1;
        R.C[1][1] = 1;
        R.C[1][0] = -1;
        R.C[2][3] = 1;
        R.C[2][2] = -1;
        v[0] = x[0] - x[2];
        v[1] = x[1] - x[0];
        v[2] = x[3] - x[2];
    }
}

// slot-space Hessian of f = d^2 accumulated into H (zero on entry), in T
template <class T>
__device__ inline void d2_hess_t(const V3* x, bool is_ee, const DistInfo& di, SMat<12, T> H) {
    Red R;
    V3 v[3];
    reduced_vars(x, is_ee, di, R, v);
    T M[9];
    if (di.type == DT_PP) {
        zero9_t(M);
        add_diag_t(M, T(2));
        scatter_block_t(H, R, 0, 0, M, T(1));
        return;
    }
    if (di.type == DT_PE) {
        V3t<T> r = to_t<T>(v[0]), e = to_t<T>(v[1]);
        T L = dot_t(e, e), s = dot_t(r, e), iL = T(1) / L;
        zero9_t(M);
        add_diag_t(M, T(2));
        outer_t(M, e, e, T(-2) * iL);
        scatter_block_t(H, R, 0, 0, M, T(1));
        T Hre[9];
        zero9_t(Hre);
        outer_t(Hre, e, r, T(-2) * iL);
        add_diag_t(Hre, T(-2) * s * iL);
        outer_t(Hre, e, e, T(4) * s * iL * iL);
        scatter_block_t(H, R, 0, 1, Hre, T(1));
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[3 * j + i] = Hre[3 * i + j];
        scatter_block_t(H, R, 1, 0, M, T(1));
        zero9_t(M);
        outer_t(M, r, r, T(-2) * iL);
        outer_t(M, r, e, T(4) * s * iL * iL);
        outer_t(M, e, r, T(4) * s * iL * iL);
        add_diag_t(M, T(2) * s * s * iL * iL);
        outer_t(M, e, e, T(-8) * s * s * iL * iL * iL);
        scatter_block_t(H, R, 1, 1, M, T(1));
        return;
    }
    // plane (PT) or line-line (EE): f = (r . (a x b))^2 / |a x b|^2.  With
    // n = a x b, N = |n|^2, s = r . n the Hessian blocks carry 1/N, s/N^2 and
    // s^2/N^3, which leave FP32's range for nearly parallel edges.  They are
    // formed in FP64 on vectors normalised by q = 1/|n| (S_k q, Ng_k q^2,
    // s q = the signed distance), so every value rounded to T is of the size
    // of the Hessian entries themselves.
    const V3 rd = v[0], ad = v[1], bd = v[2];
    const V3 nd = cross(ad, bd);
    const double Nd = dot(nd, nd), qd = 1.0 / sqrt(Nd), sh = dot(rd, nd) * qd;
    const double aad = dot(ad, ad), bbd = dot(bd, bd), abd = dot(ad, bd);
    const V3 Sd[3] = {nd, cross(bd, rd), cross(rd, ad)};
    V3t<T> Sh[3], Ngh[3];
    for (int k = 0; k < 3; ++k) Sh[k] = to_t<T>(qd * Sd[k]);
    Ngh[0] = V3t<T>{0, 0, 0};
    Ngh[1] = to_t<T>((2.0 * qd * qd) * (bbd * ad - abd * bd));
    Ngh[2] = to_t<T>((2.0 * qd * qd) * (aad * bd - abd * ad));
    const V3t<T> r = to_t<T>(rd), a = to_t<T>(ad), b = to_t<T>(bd);
    T Haa[9], Hbb[9], Hab[9];
    cross_norm_hess_t(a, b, Haa, Hbb, Hab);
    const T c2 = (T)(-2.0 * sh), c3 = (T)(2.0 * sh * sh);
    const T cs = (T)(2.0 * sh * qd), cn = (T)(-sh * sh * qd * qd);
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
            zero9_t(M);
            outer_t(M, Sh[k], Sh[l], T(2));
            outer_t(M, Sh[k], Ngh[l], c2);
            outer_t(M, Ngh[k], Sh[l], c2);
            outer_t(M, Ngh[k], Ngh[l], c3);
            if (k == 0 && l == 1) add_skew_t(M, b, -cs);
            if (k == 1 && l == 0) add_skew_t(M, b, cs);
            if (k == 0 && l == 2) add_skew_t(M, a, cs);
            if (k == 2 && l == 0) add_skew_t(M, a, -cs);
            if (k == 1 && l == 2) add_skew_t(M, r, -cs);
            if (k == 2 && l == 1) add_skew_t(M, r, cs);
            if (k == 1 && l == 1)
                for (int q = 0; q < 9; ++q) M[q] += cn * Haa[q];
            if (k == 2 && l == 2)
                for (int q = 0; q < 9; ++q) M[q] += cn * Hbb[q];
            if (k == 1 && l == 2)
                for (int q = 0; q < 9; ++q) M[q] += cn * Hab[q];
            if (k == 2 && l == 1)
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) M[3 * i + j] += cn * Hab[3 * j + i];
            scatter_block_t(H, R, k, l, M, T(1));
        }
}

// ---------------------------------------------------------------------------
// PSD projection of a translation-invariant 12x12 stencil Hessian.  Every
// barrier term depends on the four points only through their differences,
// so H = T^T K T with T (9 x 12, orthonormal rows: T[k] = -1/2 e_0 + e_{k+1}
// - 1/6 sum_{j != 0} e_j, each times I3) spanning the translation-free
// subspace, and the 12x12 projection equals T^T P(K) T with the 9x9
// K = T H T^T: the same projection with a 9x9 eigenproblem.  H is scaled by
// `scale` first; V (12x12 scratch) holds K and the projection workspace.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double tcoef(int k, int i) {  // T[k][i] for stencil slot i
    return i == 0 ? -0.5 : (i == k + 1 ? 5.0 / 6.0 : -1.0 / 6.0);
}

template <class T>
__device__ inline void project_translation_free(SMat<12, T> H, double scale, SMat<9, T> K, SMat<9, T> W, T* out) {
    // K = T (scale H) T^T, blockwise: K(k a, l b) = sum_ij T[k][i] T[l][j] H(3i + a, 3j + b)
    const T sc = (T)scale;
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    T s = 0;
                    for (int i = 0; i < 4; ++i) {
                        T r = 0;
                        for (int j = 0; j < 4; ++j) r += (T)tcoef(l, j) * H(3 * i + a, 3 * j + b);
                        s += (T)tcoef(k, i) * r;
                    }
                    K(3 * k + a, 3 * l + b) = sc * s;
                }
    psd_project<9, T>(K, W);
    // out = T^T P(K) T (row-major 12x12)
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    T s = 0;
                    for (int k = 0; k < 3; ++k) {
                        T r = 0;
                        for (int l = 0; l < 3; ++l) r += K(3 * k + a, 3 * l + b) * (T)tcoef(l, j);
                        s += (T)tcoef(k, i) * r;
                    }
                    out[12 * (3 * i + a) + 3 * j + b] = s;
                }
}

// ---------------------------------------------------------------------------
// kappa * e * b(d) for one stencil: value, gradient g12 (FP64) and the
// Hessian of e * b (without kappa, before projection) in H (12x12 slot space,
// arithmetic type T).  Returns false when d >= dhat (inactive).  eps_x <= 0
// disables the mollifier.
// ---------------------------------------------------------------------------
template <class T>
__device__ inline bool pair_barrier(const V3* x, bool is_ee, double dhat, double kappa, double eps_x,
                                    double& E, double* g12, SMat<12, T> H, bool want_h) {
    DistInfo di = classify(x, is_ee);
    double d = sqrt(di.d2);
    if (!(d < dhat)) return false;
    double gf[12];
    double f = d2_derivs(x, is_ee, di, gf, SMat<12>{nullptr, 0}, false);
    (void)f;
    double b, b1, b2;
    barrier_d012(d, dhat, b, b1, b2);
    // d(b(sqrt f)) = b1 / (2d) df ; second: b1/(2d) d2f + (b2/(4 d^2) - b1/(4 d^3)) df df^T
    double ca = b1 / (2.0 * d);
    double cb = b2 / (4.0 * d * d) - b1 / (4.0 * d * d * d);
    double gB[12];
    for (int i = 0; i < 12; ++i) gB[i] = ca * gf[i];
    if (want_h) {
        for (int i = 0; i < 12; ++i)
            for (int j = 0; j < 12; ++j) H(i, j) = T(0);
        d2_hess_t<T>(x, is_ee, di, H);
        const T cat = (T)ca, cbt = (T)cb;
        for (int i = 0; i < 12; ++i) {
            const T gi = cbt * (T)gf[i];
            for (int j = 0; j < 12; ++j) H(i, j) = cat * H(i, j) + gi * (T)gf[j];
        }
    }
    double e = 1.0;
    if (is_ee && eps_x > 0.0) {
        V3 a = x[1] - x[0], bb = x[3] - x[2];
        V3 cr = cross(a, bb);
        double c = dot(cr, cr);
        if (c < eps_x) {
            double ie = 1.0 / eps_x;
            e = c * ie * (2.0 - c * ie);
            double e1 = 2.0 * ie - 2.0 * c * ie * ie;
            double e2 = -2.0 * ie * ie;
            Red R;
            R.m = 2;
            for (int k = 0; k < 3; ++k)
                for (int i = 0; i < 4; ++i) R.C[k][i] = 0;
            R.C[0][1] = 1;
            R.C[0][0] = -1;
            R.C[1][3] = 1;
            R.C[1][2] = -1;
            V3 Na, Nb;
            double Hd[9];
            cross_norm_derivs(a, bb, Na, Nb, nullptr, Hd, Hd);
            double gc[12];
            for (int i = 0; i < 12; ++i) gc[i] = 0.0;
            scatter_grad(gc, R, 0, Na, 1.0);
            scatter_grad(gc, R, 1, Nb, 1.0);
            if (want_h) {
                // H <- e H_B + b (e2 gc gc^T + e1 d2c) + e1 (gc gB^T + gB gc^T)
                const T et = (T)e, be2 = (T)(b * e2), e1t = (T)e1;
                for (int i = 0; i < 12; ++i)
                    for (int j = 0; j < 12; ++j)
                        H(i, j) = et * H(i, j) + be2 * (T)gc[i] * (T)gc[j] +
                                  e1t * ((T)gc[i] * (T)gB[j] + (T)gB[i] * (T)gc[j]);
                T Haa[9], Hbb[9], Hab[9], Hba[9];
                cross_norm_hess_t(to_t<T>(a), to_t<T>(bb), Haa, Hbb, Hab);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) Hba[3 * j + i] = Hab[3 * i + j];
                const T be1 = (T)(b * e1);
                scatter_block_t(H, R, 0, 0, Haa, be1);
                scatter_block_t(H, R, 1, 1, Hbb, be1);
                scatter_block_t(H, R, 0, 1, Hab, be1);
                scatter_block_t(H, R, 1, 0, Hba, be1);
            }
            for (int i = 0; i < 12; ++i) gB[i] = e * gB[i] + b * e1 * gc[i];
            b = e * b;
        }
    }
    E = kappa * b;
    for (int i = 0; i < 12; ++i) g12[i] = kappa * gB[i];
    return true;
}

// energy only: kappa * e * b(d), 0 when inactive
// Squared gap between the bounding boxes of a stencil's two primitives (the
// point x0 and the triangle x1 x2 x3, or the edges x0 x1 and x2 x3): a lower
// bound of the squared distance, from differences, min and max only (a few
// FP64 operations against the hundreds of the distance classification).
__device__ __forceinline__ double stencil_box_gap2(const V3* x, bool is_ee) {
    auto axis = [&](double a0, double a1, double b0, double b1, double b2) {
        const double amin = is_ee ? fmin(a0, a1) : a0, amax = is_ee ? fmax(a0, a1) : a0;
        const double bmin = is_ee ? fmin(b1, b2) : fmin(b0, fmin(b1, b2));
        const double bmax = is_ee ? fmax(b1, b2) : fmax(b0, fmax(b1, b2));
        const double g = fmax(fmax(bmin - amax, amin - bmax), 0.0);
        return g * g;
    };
    // edges: (x0, x1) against (x2, x3); point-triangle: x0 against (x1, x2, x3)
    return axis(x[0].x, x[1].x, x[1].x, x[2].x, x[3].x) + axis(x[0].y, x[1].y, x[1].y, x[2].y, x[3].y) +
           axis(x[0].z, x[1].z, x[1].z, x[2].z, x[3].z);
}

// whether a stencil is certainly farther apart than dhat: its box gap
// exceeds dhat with a 1 % margin, far above the rounding of either
// computation, so the exact distance is at least dhat and the barrier, its
// derivatives and the active flag are all exactly zero
__device__ __forceinline__ bool stencil_beyond(const V3* x, bool is_ee, double dhat) {
    return stencil_box_gap2(x, is_ee) > 1.0201 * dhat * dhat;
}

__device__ inline double pair_barrier_energy(const V3* x, bool is_ee, double dhat, double kappa, double eps_x,
                                             double* dist_out) {
    if (!dist_out && stencil_beyond(x, is_ee, dhat)) return 0.0;
    double d2 = stencil_d2(x, is_ee);
    double d = sqrt(d2);
    if (dist_out) *dist_out = d;
    if (!(d < dhat)) return 0.0;
    if (!(d > 0.0)) return INFINITY;
    double u = d - dhat;
    double b = -u * u * log(d / dhat);
    if (is_ee && eps_x > 0.0) {
        V3 cr = cross(x[1] - x[0], x[3] - x[2]);
        double c = dot(cr, cr);
        if (c < eps_x) b *= (c / eps_x) * (2.0 - c / eps_x);
    }
    return kappa * b;
}

}  // namespace zema
