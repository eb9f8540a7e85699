/*
 * CPU oracle of the soft-rigid coupled incremental-potential-contact (IPC)
 * time step -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * this library.  It is plain, serial, FP64 code written to be checked by eye
 * against the paper; it shares no code, header, table or helper with the CUDA
 * library.  Derivatives come from second-order forward-mode dual numbers
 * (value, gradient, Hessian) applied to the plain formulas, so no derivative
 * is hand-written; pair sets come from brute force over all primitive pairs.
 *
 * What it computes, per time step and per environment (paper section III):
 *   predictor        x^ = x^t + h v^t + h^2 M^-1 f_e            (Eq. 1, Eq. 3)
 *                    q^ = q^t + h qdot^t + h^2 M_b^-1 f_e        (Eq. 2, Eq. 3)
 *   lagged friction  normal force lambda_k, closest-point weights and
 *                    normal of every pair with d < dhat at x^t   (Eq. 9, Eq. 10)
 *   Newton           minimise B_t + D (Eq. 4, Eq. 11) by projected Newton:
 *                    PSD-projected local Hessians (contact projected in the
 *                    12-dim pair space, then mapped by the coupling Jacobian,
 *                    Eq. 6-8), linear solve, convergence test, additive CCD
 *                    step bound, backtracking line search
 *   update           v = (x - x^t)/h, qdot = (q - q^t)/h         (Eq. 11)
 * plus the kinematic augmented-Lagrangian term (Eq. 13) for kinematic affine
 * bodies.
 *
 * Readings of points the paper leaves open (all shared with the CUDA path as
 * mathematics, never as code):
 *   d in b(d) is the unsigned Euclidean distance (Eq. 5);
 *   Neo-Hookean Psi = mu/2 (tr F^T F - 3) - mu ln J + lambda/2 (ln J)^2, +inf
 *   for J <= 0, its 9x9 F-space Hessian projected to PSD;
 *   affine orthogonality Hessian (9x9 in A) projected to PSD;
 *   edge-edge barrier multiplied by the IPC mollifier e(c), c = |ea x eb|^2,
 *   eps_x = 1e-3 |ea_rest|^2 |eb_rest|^2;
 *   friction: lagged once per step at x^t, lambda = kappa e |b'(d)|, tangent
 *   operator I - n n^T, f0 the cubic with f0' = f1 and f0(eps_v h) = eps_v h;
 *   pair mu = min of the two bodies' mu;
 *   kappa adaptive: kappa_min = 1e3 * mean soft lumped mass (or mean affine
 *   mass / 8), initial value from gradient balance clamped to [1, 100] x
 *   kappa_min, doubled (capped at 1e4 x kappa_min) when d_min < 0.1 dhat and
 *   d_min decreased over the step;
 *   Newton stop: max abs component of the step over soft vertices and over
 *   the affine bodies' mesh vertices (J p_b) <= tol_rel * bbox_diag * h; the
 *   step that meets the tolerance is not applied;
 *   line search: alpha starts at the ACCD bound over pairs whose swept AABBs,
 *   inflated by dhat/2, overlap (s = 0.1, t_c = 1), halved until
 *   E(x + alpha p) <= E(x), at most 60 halvings;
 *   kinematic AL: kappa_A = 1e3 m_b, multiplier update after Newton converges
 *   when max |q - q~| > tol, at most max_al_rounds rounds.
 *
 * Pins: the paper prints no worked example or trajectory, so no stored value
 * comes from it.  Every function here is pinned instead by mathematics in the
 * tests: closed forms, brute force, finite differences and invariants.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <string>
#include <tuple>
#include <array>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

// Loops whose iterations write only their own slots run in parallel when the
// library is built with OpenMP; every sum over them is then taken serially,
// in index order, afterwards, so results are bit-identical to a serial run
// for any thread count.
// The thread count is the library's own (orc_set_threads, 1 at load), so
// the process-wide OpenMP setting of other libraries is left alone.
static int g_orc_threads = 1;
#ifdef _OPENMP
#define ORC_PRAGMA(x) _Pragma(#x)
#define ORC_PARALLEL_FOR ORC_PRAGMA(omp parallel for schedule(static) num_threads(g_orc_threads))
#define ORC_PARALLEL_FOR_DYNAMIC ORC_PRAGMA(omp parallel for schedule(dynamic, 8) num_threads(g_orc_threads))
#else
#define ORC_PARALLEL_FOR
#define ORC_PARALLEL_FOR_DYNAMIC
#endif

namespace {

const double INF = std::numeric_limits<double>::infinity();

// ===========================================================================
// Second-order forward-mode dual numbers: value, gradient and Hessian with
// respect to N independent variables.
// ===========================================================================
template <int N>
struct D2 {
    double v;
    double g[N];
    double h[N][N];
};

template <int N>
D2<N> cst(double c) {
    D2<N> r;
    r.v = c;
    for (int i = 0; i < N; ++i) {
        r.g[i] = 0.0;
        for (int j = 0; j < N; ++j) r.h[i][j] = 0.0;
    }
    return r;
}

template <int N>
D2<N> var(double c, int k) {
    D2<N> r = cst<N>(c);
    r.g[k] = 1.0;
    return r;
}

template <int N>
D2<N> operator+(const D2<N>& a, const D2<N>& b) {
    D2<N> r;
    r.v = a.v + b.v;
    for (int i = 0; i < N; ++i) {
        r.g[i] = a.g[i] + b.g[i];
        for (int j = 0; j < N; ++j) r.h[i][j] = a.h[i][j] + b.h[i][j];
    }
    return r;
}

template <int N>
D2<N> operator-(const D2<N>& a, const D2<N>& b) {
    D2<N> r;
    r.v = a.v - b.v;
    for (int i = 0; i < N; ++i) {
        r.g[i] = a.g[i] - b.g[i];
        for (int j = 0; j < N; ++j) r.h[i][j] = a.h[i][j] - b.h[i][j];
    }
    return r;
}

template <int N>
D2<N> operator*(double s, const D2<N>& a) {
    D2<N> r;
    r.v = s * a.v;
    for (int i = 0; i < N; ++i) {
        r.g[i] = s * a.g[i];
        for (int j = 0; j < N; ++j) r.h[i][j] = s * a.h[i][j];
    }
    return r;
}

template <int N>
D2<N> operator*(const D2<N>& a, double s) {
    return s * a;
}

template <int N>
D2<N> operator+(const D2<N>& a, double c) {
    D2<N> r = a;
    r.v += c;
    return r;
}

template <int N>
D2<N> operator*(const D2<N>& a, const D2<N>& b) {
    D2<N> r;
    r.v = a.v * b.v;
    for (int i = 0; i < N; ++i) {
        r.g[i] = a.v * b.g[i] + b.v * a.g[i];
        for (int j = 0; j < N; ++j)
            r.h[i][j] = a.v * b.h[i][j] + b.v * a.h[i][j] + a.g[i] * b.g[j] + b.g[i] * a.g[j];
    }
    return r;
}

// r = f(a) given f(a.v), f'(a.v), f''(a.v)
template <int N>
D2<N> chain(const D2<N>& a, double f, double f1, double f2) {
    D2<N> r;
    r.v = f;
    for (int i = 0; i < N; ++i) {
        r.g[i] = f1 * a.g[i];
        for (int j = 0; j < N; ++j) r.h[i][j] = f1 * a.h[i][j] + f2 * a.g[i] * a.g[j];
    }
    return r;
}

template <int N>
D2<N> inv(const D2<N>& a) {
    double y = a.v;
    return chain(a, 1.0 / y, -1.0 / (y * y), 2.0 / (y * y * y));
}

template <int N>
D2<N> operator/(const D2<N>& a, const D2<N>& b) {
    return a * inv(b);
}

template <int N>
D2<N> dsqrt(const D2<N>& a) {
    double s = std::sqrt(a.v);
    return chain(a, s, 0.5 / s, -0.25 / (s * a.v));
}

template <int N>
D2<N> dlog(const D2<N>& a) {
    return chain(a, std::log(a.v), 1.0 / a.v, -1.0 / (a.v * a.v));
}

template <int N>
struct V3 {
    D2<N> c[3];
};

template <int N>
V3<N> vsub(const V3<N>& a, const V3<N>& b) {
    V3<N> r;
    for (int i = 0; i < 3; ++i) r.c[i] = a.c[i] - b.c[i];
    return r;
}

template <int N>
D2<N> vdot(const V3<N>& a, const V3<N>& b) {
    return a.c[0] * b.c[0] + a.c[1] * b.c[1] + a.c[2] * b.c[2];
}

template <int N>
V3<N> vcross(const V3<N>& a, const V3<N>& b) {
    V3<N> r;
    r.c[0] = a.c[1] * b.c[2] - a.c[2] * b.c[1];
    r.c[1] = a.c[2] * b.c[0] - a.c[0] * b.c[2];
    r.c[2] = a.c[0] * b.c[1] - a.c[1] * b.c[0];
    return r;
}

// point k of a 12-variable stencil (4 points) as dual numbers
V3<12> point_var(const double* x12, int k) {
    V3<12> r;
    for (int i = 0; i < 3; ++i) r.c[i] = var<12>(x12[3 * k + i], 3 * k + i);
    return r;
}

// ===========================================================================
// Plain double 3-vectors
// ===========================================================================
struct P3 {
    double x, y, z;
};
P3 p3(const double* a) { return P3{a[0], a[1], a[2]}; }
P3 sub(P3 a, P3 b) { return P3{a.x - b.x, a.y - b.y, a.z - b.z}; }
P3 add(P3 a, P3 b) { return P3{a.x + b.x, a.y + b.y, a.z + b.z}; }
P3 mul(double s, P3 a) { return P3{s * a.x, s * a.y, s * a.z}; }
double dot(P3 a, P3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
P3 cross(P3 a, P3 b) { return P3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }

// ===========================================================================
// Symmetric eigen-decomposition by cyclic Jacobi rotations and PSD projection
// ===========================================================================
// A (n x n, row-major) is overwritten; evals (n), evecs (n x n, columns).
void jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& evals, std::vector<double>& V) {
    V.assign(n * n, 0.0);
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += A[i * n + j] * A[i * n + j];
                if (i != j) off += A[i * n + j] * A[i * n + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double app = A[p * n + p], aqq = A[q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                // A <- R^T A R with rotation in the (p, q) plane
                for (int k = 0; k < n; ++k) {
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    evals.resize(n);
    for (int i = 0; i < n; ++i) evals[i] = A[i * n + i];
}

// Replace symmetric H (n x n) by V max(Lambda, 0) V^T.
void psd_project(int n, double* H) {
    std::vector<double> A(H, H + n * n), ev, V;
    // symmetrise first
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) {
            double m = 0.5 * (A[i * n + j] + A[j * n + i]);
            A[i * n + j] = A[j * n + i] = m;
        }
    jacobi_eigen(n, A, ev, V);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k)
                if (ev[k] > 0.0) s += V[i * n + k] * ev[k] * V[j * n + k];
            H[i * n + j] = s;
        }
}

// ===========================================================================
// Barrier (Eq. 5), friction mollifier f0/f1 (Eq. 10)
// ===========================================================================
double barrier(double d, double dhat) {
    if (d <= 0.0) return INF;
    if (d >= dhat) return 0.0;
    return -(d - dhat) * (d - dhat) * std::log(d / dhat);
}

// derivative of b with respect to d (used for the lagged normal force)
double barrier_d1(double d, double dhat) {
    if (d >= dhat) return 0.0;
    return -2.0 * (d - dhat) * std::log(d / dhat) - (d - dhat) * (d - dhat) / d;
}

// f0 with f0' = f1 (Eq. 10) and f0(eps_v h) = eps_v h
double f0(double y, double eh) {
    if (y >= eh) return y;
    return -y * y * y / (3.0 * eh * eh) + y * y / eh + eh / 3.0;
}
double f1(double y, double eh) {
    if (y >= eh) return 1.0;
    return -y * y / (eh * eh) + 2.0 * y / eh;
}

// ===========================================================================
// Distances by enumeration of closest-feature candidates (no region
// classifier): the distance between a point and a triangle, or between two
// segments, is the smallest of the candidate distances whose closest points
// lie in the interior of their features, plus all vertex-vertex candidates.
// Type codes: which feature pair realised the minimum.
// ===========================================================================
enum Kind { K_PP = 0, K_PE = 1, K_PT = 2, K_EE = 3 };

struct Cand {
    double d2;
    int kind;
    int a[4];  // stencil slot indices of the points that take part
    int na;
    double w[4];  // closest-point weights for Delta = sum w_i x_i over slots a[]
};

// point-segment: candidate for segment interior only
bool seg_interior(P3 p, P3 e0, P3 e1, double& d2, double& t) {
    P3 e = sub(e1, e0);
    double ee = dot(e, e);
    if (ee <= 0.0) return false;
    t = dot(sub(p, e0), e) / ee;
    if (!(t > 0.0 && t < 1.0)) return false;
    P3 c = sub(p, add(e0, mul(t, e)));
    d2 = dot(c, c);
    return true;
}

// Enumerate PT candidates for stencil (p, t0, t1, t2) = slots (0, 1, 2, 3).
Cand pt_closest(const double* x12) {
    P3 p = p3(x12), t[3] = {p3(x12 + 3), p3(x12 + 6), p3(x12 + 9)};
    Cand best;
    best.d2 = INF;
    // vertex-vertex
    for (int i = 0; i < 3; ++i) {
        P3 d = sub(p, t[i]);
        double d2 = dot(d, d);
        if (d2 < best.d2) {
            best = Cand{d2, K_PP, {0, 1 + i, 0, 0}, 2, {1.0, -1.0, 0, 0}};
        }
    }
    // point-edge interiors
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3;
        double d2, s;
        if (seg_interior(p, t[i], t[j], d2, s) && d2 < best.d2)
            best = Cand{d2, K_PE, {0, 1 + i, 1 + j, 0}, 3, {1.0, -(1.0 - s), -s, 0}};
    }
    // triangle interior
    P3 n = cross(sub(t[1], t[0]), sub(t[2], t[0]));
    double nn = dot(n, n);
    if (nn > 0.0) {
        P3 r = sub(p, t[0]);
        double h = dot(r, n);
        P3 q = sub(r, mul(h / nn, n));  // projection relative to t0
        // barycentric coordinates of the projection
        P3 e1 = sub(t[1], t[0]), e2 = sub(t[2], t[0]);
        double d11 = dot(e1, e1), d12 = dot(e1, e2), d22 = dot(e2, e2);
        double q1 = dot(q, e1), q2 = dot(q, e2);
        double den = d11 * d22 - d12 * d12;
        if (den > 0.0) {
            double b1 = (d22 * q1 - d12 * q2) / den;
            double b2 = (d11 * q2 - d12 * q1) / den;
            double b0 = 1.0 - b1 - b2;
            if (b0 > 0.0 && b1 > 0.0 && b2 > 0.0) {
                double d2 = h * h / nn;
                if (d2 < best.d2) best = Cand{d2, K_PT, {0, 1, 2, 3}, 4, {1.0, -b0, -b1, -b2}};
            }
        }
    }
    return best;
}

// Enumerate EE candidates for stencil (ea0, ea1, eb0, eb1) = slots (0,1,2,3).
Cand ee_closest(const double* x12) {
    P3 a0 = p3(x12), a1 = p3(x12 + 3), b0 = p3(x12 + 6), b1 = p3(x12 + 9);
    P3 pts[4] = {a0, a1, b0, b1};
    Cand best;
    best.d2 = INF;
    // vertex-vertex: endpoint of a with endpoint of b
    for (int i = 0; i < 2; ++i)
        for (int j = 2; j < 4; ++j) {
            P3 d = sub(pts[i], pts[j]);
            double d2 = dot(d, d);
            if (d2 < best.d2) best = Cand{d2, K_PP, {i, j, 0, 0}, 2, {1.0, -1.0, 0, 0}};
        }
    // endpoint of one edge against the interior of the other
    for (int i = 0; i < 4; ++i) {
        int o0 = (i < 2) ? 2 : 0, o1 = o0 + 1;
        double d2, s;
        if (seg_interior(pts[i], pts[o0], pts[o1], d2, s) && d2 < best.d2) {
            // Delta = x_i - ((1-s) x_o0 + s x_o1) for an endpoint of a; sign flips for b
            double sg = (i < 2) ? 1.0 : -1.0;
            best = Cand{d2, K_PE, {i, o0, o1, 0}, 3, {sg, -sg * (1.0 - s), -sg * s, 0}};
        }
    }
    // interior-interior (non-parallel lines)
    P3 ea = sub(a1, a0), eb = sub(b1, b0);
    P3 n = cross(ea, eb);
    double nn = dot(n, n);
    if (nn > 1e-20 * dot(ea, ea) * dot(eb, eb)) {
        P3 r = sub(a0, b0);
        // closest parameters of the two lines
        double a = dot(ea, ea), b = dot(ea, eb), c = dot(eb, eb), d = dot(ea, r), e = dot(eb, r);
        double den = a * c - b * b;
        double s = (b * e - c * d) / den;
        double t = (a * e - b * d) / den;
        if (s > 0.0 && s < 1.0 && t > 0.0 && t < 1.0) {
            double hh = dot(r, n);
            double d2 = hh * hh / nn;
            if (d2 < best.d2) best = Cand{d2, K_EE, {0, 1, 2, 3}, 4, {1.0 - s, s, -(1.0 - t), -t}};
        }
    }
    return best;
}

// Squared distance of the chosen candidate as a dual number over the 12
// stencil coordinates.
D2<12> cand_d2(const double* x12, const Cand& c, bool is_ee) {
    if (c.kind == K_PP) {
        V3<12> a = point_var(x12, c.a[0]), b = point_var(x12, c.a[1]);
        V3<12> d = vsub(a, b);
        return vdot(d, d);
    }
    if (c.kind == K_PE) {
        V3<12> p = point_var(x12, c.a[0]), e0 = point_var(x12, c.a[1]), e1 = point_var(x12, c.a[2]);
        V3<12> cr = vcross(vsub(e0, p), vsub(e1, p));
        V3<12> e = vsub(e1, e0);
        return vdot(cr, cr) / vdot(e, e);
    }
    // plane / line-line: ((x_a - x_b) . n)^2 / |n|^2
    V3<12> q0 = point_var(x12, 0), q1 = point_var(x12, 1), q2 = point_var(x12, 2), q3 = point_var(x12, 3);
    V3<12> n, r;
    if (!is_ee) {
        n = vcross(vsub(q2, q1), vsub(q3, q1));
        r = vsub(q0, q1);
    } else {
        n = vcross(vsub(q1, q0), vsub(q3, q2));
        r = vsub(q0, q2);
    }
    D2<12> h = vdot(r, n);
    return (h * h) / vdot(n, n);
}

double stencil_d2(const double* x12, bool is_ee) {
    return is_ee ? ee_closest(x12).d2 : pt_closest(x12).d2;
}

// IPC edge-edge mollifier e(c), c = |ea x eb|^2 (dual number)
D2<12> ee_mollifier(const double* x12, double eps_x) {
    V3<12> q0 = point_var(x12, 0), q1 = point_var(x12, 1), q2 = point_var(x12, 2), q3 = point_var(x12, 3);
    V3<12> cr = vcross(vsub(q1, q0), vsub(q3, q2));
    D2<12> c = vdot(cr, cr);
    if (c.v >= eps_x) return cst<12>(1.0);
    D2<12> r = (1.0 / eps_x) * c;
    return r * (cst<12>(2.0) - r);
}

double ee_mollifier_value(const double* x12, double eps_x) {
    P3 cr = cross(sub(p3(x12 + 3), p3(x12)), sub(p3(x12 + 9), p3(x12 + 6)));
    double c = dot(cr, cr);
    if (c >= eps_x) return 1.0;
    double r = c / eps_x;
    return r * (2.0 - r);
}

// Barrier energy of one pair (without kappa) with gradient and Hessian in the
// 12-dim stencil space.  Returns false when the pair is inactive (d >= dhat).
bool pair_barrier(const double* x12, bool is_ee, double dhat, double eps_x, D2<12>& out) {
    Cand c = is_ee ? ee_closest(x12) : pt_closest(x12);
    double d = std::sqrt(c.d2);
    if (!(d < dhat)) return false;
    D2<12> dd = dsqrt(cand_d2(x12, c, is_ee));
    D2<12> u = dd + (-dhat);
    D2<12> b = (-1.0) * (u * u) * dlog((1.0 / dhat) * dd);
    if (is_ee) b = ee_mollifier(x12, eps_x) * b;
    out = b;
    return true;
}

// ===========================================================================
// Neo-Hookean energy density in F-space (9 variables, F row-major)
// ===========================================================================
bool nh_psi(const double* F9, double mu, double lam, D2<9>& out) {
    D2<9> F[9];
    for (int i = 0; i < 9; ++i) F[i] = var<9>(F9[i], i);
    D2<9> J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
              F[2] * (F[3] * F[7] - F[4] * F[6]);
    if (!(J.v > 0.0)) return false;
    D2<9> tr = cst<9>(0.0);
    for (int i = 0; i < 9; ++i) tr = tr + F[i] * F[i];
    D2<9> lj = dlog(J);
    out = (0.5 * mu) * (tr + (-3.0)) - mu * lj + (0.5 * lam) * (lj * lj);
    return true;
}

// St. Venant-Kirchhoff energy density in F-space: Green strain
// E = (F^T F - I) / 2, Psi = mu E:E + lambda/2 tr(E)^2 (finite for every F)
D2<9> stvk_psi(const double* F9, double mu, double lam) {
    D2<9> F[9];
    for (int i = 0; i < 9; ++i) F[i] = var<9>(F9[i], i);
    D2<9> ee = cst<9>(0.0), tr = cst<9>(0.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            D2<9> c = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
            D2<9> Eij = 0.5 * (c + (i == j ? -1.0 : 0.0));
            ee = ee + Eij * Eij;
            if (i == j) tr = tr + Eij;
        }
    return mu * ee + (0.5 * lam) * (tr * tr);
}

// Fixed-corotated energy density: Psi = mu |F - R|^2 + lambda/2 (J - 1)^2
// with R the rotation of the polar decomposition F = R S, computed by
// Newton's iteration R <- (R + R^-T)/2 from R = F carried out on dual numbers
// (so the derivatives of R are those of the converged iteration); J <= 0 is
// not admitted (false), so R is a proper rotation.
bool fcr_psi(const double* F9, double mu, double lam, D2<9>& out) {
    D2<9> F[9];
    for (int i = 0; i < 9; ++i) F[i] = var<9>(F9[i], i);
    auto det3 = [](const D2<9>* A) {
        return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
               A[2] * (A[3] * A[7] - A[4] * A[6]);
    };
    D2<9> J = det3(F);
    if (!(J.v > 0.0)) return false;
    D2<9> R[9];
    for (int i = 0; i < 9; ++i) R[i] = F[i];
    int extra = -1;
    for (int it = 0; it < 80 && extra != 0; ++it) {
        // R^-T = cof(R) / det(R)
        D2<9> Cf[9] = {R[4] * R[8] - R[5] * R[7], R[5] * R[6] - R[3] * R[8], R[3] * R[7] - R[4] * R[6],
                       R[2] * R[7] - R[1] * R[8], R[0] * R[8] - R[2] * R[6], R[1] * R[6] - R[0] * R[7],
                       R[1] * R[5] - R[2] * R[4], R[2] * R[3] - R[0] * R[5], R[0] * R[4] - R[1] * R[3]};
        D2<9> d = det3(R);
        double diff = 0.0;
        for (int i = 0; i < 9; ++i) {
            D2<9> r = 0.5 * (R[i] + Cf[i] / d);
            diff = std::max(diff, std::fabs(r.v - R[i].v));
            R[i] = r;
        }
        // a few more iterations once the value has converged, for the
        // derivative parts
        if (extra < 0 && diff < 1e-15) extra = 4;
        if (extra > 0) --extra;
    }
    D2<9> s = cst<9>(0.0);
    for (int i = 0; i < 9; ++i) {
        D2<9> e = F[i] - R[i];
        s = s + e * e;
    }
    D2<9> jm = J + (-1.0);
    out = mu * s + (0.5 * lam) * (jm * jm);
    return true;
}

// Affine orthogonality energy |A A^T - I|_F^2 (9 variables, A row-major)
D2<9> ortho(const double* A9) {
    D2<9> A[9];
    for (int i = 0; i < 9; ++i) A[i] = var<9>(A9[i], i);
    D2<9> s = cst<9>(0.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            D2<9> m = A[3 * i] * A[3 * j] + A[3 * i + 1] * A[3 * j + 1] + A[3 * i + 2] * A[3 * j + 2];
            if (i == j) m = m + (-1.0);
            s = s + m * m;
        }
    return s;
}

// ===========================================================================
// Scene
// ===========================================================================
struct Params {
    double dt, dhat, kappa, eps_v, tol_rel, g[3], pcg_rel_tol;
    int max_newton, max_al_rounds;
    int al_extrapolate;  // start each step's kinematic multipliers at 2 lambda^t - lambda^(t-1)
};

struct Affine {
    int env, mode;  // 0 dynamic, 1 fixed, 2 kinematic
    std::vector<double> V;  // rest vertices (nv x 3), caller's frame
    std::vector<int> F;
    double rho, stiffness, mu;
    double q[12], qd[12], qt[12], qhat[12], qtarget[12], lamA[12];
    double lamA_prev[12];  // the multipliers at the end of the step before the last one
    double M[144];
    double m, vol;
    int sv0;  // first surface vertex
};

// Prismatic joint between two affine bodies, constants at the initial state
// in the caller's frame (x = A y + p): B_b = A_b(0)^-1, y_b the joint point
// (body 1's initial centre of mass) in body b's rest frame, d1 the axis in
// body 1's rest frame.
struct Joint {
    int a1, a2, env;
    double kappa;
    double B1[9], B2[9], y1[3], y2[3], d1[3];
    double lam[12];
};

struct SoftBody {
    int env, v0, nv, t0, nt;
    double mu_l, lam_l, mu, rho;
    int model = 0;  // 0 Neo-Hookean, 1 St. Venant-Kirchhoff, 2 fixed corotated
};

struct SV {
    int body;     // global body id
    int affine;   // 1 if on an affine body
    int idx;      // soft: global vertex; affine: local vertex of that body
};

struct Lagged {
    int is_ee;
    int s[4];        // surface vertices (EE: a0 a1 b0 b1, PT: p t0 t1 t2)
    double w[4];     // Delta = sum w_i (x_i - x_i^t)
    double n[3];     // unit normal at x^t
    double lam, mu;  // lagged normal force, friction coefficient
};

struct Pair {
    int is_ee;
    int s[4];
};

struct StepStats {
    double newton_iters, ls_halvings, al_rounds, n_active, dmin, energy, kappa, status, warm_accepted;
};

struct Scene {
    Params P;
    int n_envs = 1;
    // soft
    std::vector<double> X, x, v, xt, xhat, mass;
    std::vector<double> spring_k, spring_x;  // per soft vertex: spring stiffness (0: none) and target
    std::vector<int> tets, vert_body;
    std::vector<double> Dminv, tvol;
    std::vector<int> tet_body;
    std::vector<SoftBody> soft;
    // affine
    std::vector<Affine> aff;
    std::vector<Joint> joints;
    // bodies: global id -> (kind, index)
    std::vector<std::pair<int, int>> bodies;
    // surface
    std::vector<SV> sv;
    std::vector<int> edges, tris;  // surface vertex indices
    std::vector<double> edge_rest_len2;
    // per env
    std::vector<double> kappa, kappa_min, dmin_last, diag;
    std::vector<int> kappa_init;
    std::vector<std::vector<Lagged>> lagged;
    bool finalized = false;
    std::string err;
    std::vector<StepStats> stats;
    std::vector<double> energy_log;  // energy at every Newton iterate (env-level)
};

int body_env(const Scene& S, int b) {
    auto bk = S.bodies[b];
    return bk.first == 0 ? S.soft[bk.second].env : S.aff[bk.second].env;
}
// 0 soft, 1 affine dynamic, 2 fixed, 3 kinematic
int body_class(const Scene& S, int b) {
    auto bk = S.bodies[b];
    if (bk.first == 0) return 0;
    int m = S.aff[bk.second].mode;
    return m == 0 ? 1 : (m == 1 ? 2 : 3);
}
double body_mu(const Scene& S, int b) {
    auto bk = S.bodies[b];
    return bk.first == 0 ? S.soft[bk.second].mu : S.aff[bk.second].mu;
}

// World position of a surface vertex for soft positions xs and affine states qs
P3 sv_pos(const Scene& S, int s, const std::vector<double>& xs, const std::vector<double>& qs) {
    const SV& v = S.sv[s];
    if (!v.affine) return p3(&xs[3 * v.idx]);
    int a = S.bodies[v.body].second;
    const double* q = &qs[12 * a];
    const double* x0 = &S.aff[a].V[3 * v.idx];
    // x = A x0 + p with A = (a1, a2, a3)^T (rows)
    P3 r;
    r.x = q[0] + q[3] * x0[0] + q[4] * x0[1] + q[5] * x0[2];
    r.y = q[1] + q[6] * x0[0] + q[7] * x0[1] + q[8] * x0[2];
    r.z = q[2] + q[9] * x0[0] + q[10] * x0[1] + q[11] * x0[2];
    return r;
}

// ---------------------------------------------------------------------------
// Per-environment DOF layout: soft vertices of the env (3 each) in global
// order, then the env's non-fixed affine bodies (12 each, (p, a1, a2, a3)).
// ---------------------------------------------------------------------------
struct EnvDofs {
    int n = 0;
    std::vector<int> vert_dof;  // global soft vertex -> dof offset or -1
    std::vector<int> aff_dof;   // affine index -> dof offset or -1
    std::vector<int> verts, affs;
};

EnvDofs env_dofs(const Scene& S, int env) {
    EnvDofs D;
    D.vert_dof.assign(S.x.size() / 3, -1);
    D.aff_dof.assign(S.aff.size(), -1);
    for (size_t i = 0; i < S.vert_body.size(); ++i)
        if (body_env(S, S.vert_body[i]) == env) {
            D.vert_dof[i] = D.n;
            D.verts.push_back((int)i);
            D.n += 3;
        }
    for (size_t a = 0; a < S.aff.size(); ++a)
        if (S.aff[a].env == env && S.aff[a].mode != 1) {
            D.aff_dof[a] = D.n;
            D.affs.push_back((int)a);
            D.n += 12;
        }
    return D;
}

// Jacobian of a surface vertex position with respect to the env DOFs:
// returns the number of DOFs (0, 3 or 12), their first offset and J (3 x 12).
int sv_jac(const Scene& S, const EnvDofs& D, int s, int& off, double J[3][12]) {
    const SV& v = S.sv[s];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 12; ++j) J[i][j] = 0.0;
    if (!v.affine) {
        off = D.vert_dof[v.idx];
        if (off < 0) return 0;
        for (int i = 0; i < 3; ++i) J[i][i] = 1.0;
        return 3;
    }
    int a = S.bodies[v.body].second;
    off = D.aff_dof[a];
    if (off < 0) return 0;
    const double* x0 = &S.aff[a].V[3 * v.idx];
    // d x_i / d p_i = 1 ; d x_i / d (a_i)_k = x0_k
    for (int i = 0; i < 3; ++i) {
        J[i][i] = 1.0;
        for (int k = 0; k < 3; ++k) J[i][3 + 3 * i + k] = x0[k];
    }
    return 12;
}

// ---------------------------------------------------------------------------
// Pair validity (which pairs belong to the contact set C)
// ---------------------------------------------------------------------------
bool pair_valid(const Scene& S, int sa, int sb) {
    int ba = S.sv[sa].body, bb = S.sv[sb].body;
    if (body_env(S, ba) != body_env(S, bb)) return false;
    int ca = body_class(S, ba), cb = body_class(S, bb);
    if ((ca == 2 || ca == 3) && (cb == 2 || cb == 3)) return false;  // both fixed / kinematic
    if (ba == bb && ca != 0) return false;  // same affine body
    return true;
}

bool pt_valid(const Scene& S, int p, const int* t) {
    if (p == t[0] || p == t[1] || p == t[2]) return false;
    return pair_valid(S, p, t[0]);
}
bool ee_valid(const Scene& S, const int* ea, const int* eb) {
    if (ea[0] == eb[0] || ea[0] == eb[1] || ea[1] == eb[0] || ea[1] == eb[1]) return false;
    return pair_valid(S, ea[0], eb[0]);
}

struct Box {
    double lo[3], hi[3];
};
Box box_of(const std::vector<P3>& P, const int* ids, int n, double infl) {
    Box b;
    b.lo[0] = b.hi[0] = P[ids[0]].x;
    b.lo[1] = b.hi[1] = P[ids[0]].y;
    b.lo[2] = b.hi[2] = P[ids[0]].z;
    for (int i = 1; i < n; ++i) {
        const P3& p = P[ids[i]];
        b.lo[0] = std::min(b.lo[0], p.x); b.hi[0] = std::max(b.hi[0], p.x);
        b.lo[1] = std::min(b.lo[1], p.y); b.hi[1] = std::max(b.hi[1], p.y);
        b.lo[2] = std::min(b.lo[2], p.z); b.hi[2] = std::max(b.hi[2], p.z);
    }
    for (int k = 0; k < 3; ++k) {
        b.lo[k] -= infl;
        b.hi[k] += infl;
    }
    return b;
}
Box box_union(const Box& a, const Box& b) {
    Box r;
    for (int k = 0; k < 3; ++k) {
        r.lo[k] = std::min(a.lo[k], b.lo[k]);
        r.hi[k] = std::max(a.hi[k], b.hi[k]);
    }
    return r;
}
bool overlap(const Box& a, const Box& b) {
    for (int k = 0; k < 3; ++k)
        if (a.lo[k] > b.hi[k] || b.lo[k] > a.hi[k]) return false;
    return true;
}

void all_sv_pos(const Scene& S, const std::vector<double>& xs, const std::vector<double>& qs, std::vector<P3>& P) {
    P.resize(S.sv.size());
    for (size_t s = 0; s < S.sv.size(); ++s) P[s] = sv_pos(S, (int)s, xs, qs);
}

// All valid pairs of env `env` whose AABBs (inflated by dhat/2 per side)
// overlap.  With P1 != nullptr the boxes span both P0 and P1 (swept).
void candidate_pairs(const Scene& S, int env, const std::vector<P3>& P0, const std::vector<P3>* P1,
                     std::vector<Pair>& out) {
    out.clear();
    double infl = 0.5 * S.P.dhat;
    size_t nt = S.tris.size() / 3, ne = S.edges.size() / 2, ns = S.sv.size();
    auto bx = [&](const int* ids, int n) {
        Box b = box_of(P0, ids, n, infl);
        if (P1) b = box_union(b, box_of(*P1, ids, n, infl));
        return b;
    };
    std::vector<Box> tb(nt), eb(ne), pb(ns);
    ORC_PARALLEL_FOR
    for (long t = 0; t < (long)nt; ++t) tb[t] = bx(&S.tris[3 * t], 3);
    ORC_PARALLEL_FOR
    for (long e = 0; e < (long)ne; ++e) eb[e] = bx(&S.edges[2 * e], 2);
    ORC_PARALLEL_FOR
    for (long s = 0; s < (long)ns; ++s) {
        int id = (int)s;
        pb[s] = bx(&id, 1);
    }
    // every query primitive's pairs go to a list of its own, concatenated in
    // query order afterwards: the same list, in the same order, whatever the
    // thread count
    std::vector<std::vector<Pair>> lp(ns), le(ne);
    ORC_PARALLEL_FOR_DYNAMIC
    for (long s = 0; s < (long)ns; ++s) {
        if (body_env(S, S.sv[s].body) != env) continue;
        for (size_t t = 0; t < nt; ++t) {
            const int* T = &S.tris[3 * t];
            if (!pt_valid(S, (int)s, T)) continue;
            if (!overlap(pb[s], tb[t])) continue;
            lp[s].push_back(Pair{0, {(int)s, T[0], T[1], T[2]}});
        }
    }
    ORC_PARALLEL_FOR_DYNAMIC
    for (long a = 0; a < (long)ne; ++a) {
        const int* A = &S.edges[2 * a];
        if (body_env(S, S.sv[A[0]].body) != env) continue;
        for (size_t b = a + 1; b < ne; ++b) {
            const int* B = &S.edges[2 * b];
            if (!ee_valid(S, A, B)) continue;
            if (!overlap(eb[a], eb[b])) continue;
            le[a].push_back(Pair{1, {A[0], A[1], B[0], B[1]}});
        }
    }
    for (const auto& l : lp) out.insert(out.end(), l.begin(), l.end());
    for (const auto& l : le) out.insert(out.end(), l.begin(), l.end());
}

void stencil(const std::vector<P3>& P, const Pair& pr, double* x12) {
    for (int k = 0; k < 4; ++k) {
        x12[3 * k] = P[pr.s[k]].x;
        x12[3 * k + 1] = P[pr.s[k]].y;
        x12[3 * k + 2] = P[pr.s[k]].z;
    }
}

double ee_eps_x(const Scene& S, const Pair& pr) {
    // rest-length based threshold; the edge rest lengths are looked up by the
    // surface-vertex rest positions
    auto rest = [&](int s) -> P3 {
        const SV& v = S.sv[s];
        if (!v.affine) return p3(&S.X[3 * v.idx]);
        return p3(&S.aff[S.bodies[v.body].second].V[3 * v.idx]);
    };
    P3 a = sub(rest(pr.s[1]), rest(pr.s[0])), b = sub(rest(pr.s[3]), rest(pr.s[2]));
    return 1e-3 * dot(a, a) * dot(b, b);
}

// ===========================================================================
// Linear algebra on the env system
// ===========================================================================
struct Trip {
    int i, j;
    double v;
};

struct Sys {
    int n;
    std::vector<double> g;
    std::vector<Trip> H;
};

// add a local block: DOF ranges (offa, na) x (offb, nb), values M (na x nb)
void add_block(Sys& Y, int offa, int na, int offb, int nb, const double* M, int ld) {
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j) {
            double v = M[i * ld + j];
            if (v != 0.0) Y.H.push_back(Trip{offa + i, offb + j, v});
        }
}

// Dense Cholesky solve (n small): returns false if not positive definite.
bool dense_solve(int n, const std::vector<Trip>& T, const std::vector<double>& b, std::vector<double>& x) {
    std::vector<double> A((size_t)n * n, 0.0);
    for (const Trip& t : T) A[(size_t)t.i * n + t.j] += t.v;
    for (int j = 0; j < n; ++j) {
        double s = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(s > 0.0)) return false;
        double l = std::sqrt(s);
        A[(size_t)j * n + j] = l;
        ORC_PARALLEL_FOR
        for (int i = j + 1; i < n; ++i) {
            double t = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = t / l;
        }
    }
    x = b;
    for (int i = 0; i < n; ++i) {
        double t = x[i];
        for (int k = 0; k < i; ++k) t -= A[(size_t)i * n + k] * x[k];
        x[i] = t / A[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double t = x[i];
        for (int k = i + 1; k < n; ++k) t -= A[(size_t)k * n + i] * x[k];
        x[i] = t / A[(size_t)i * n + i];
    }
    return true;
}

// Invert a small square matrix (Gauss-Jordan with partial pivoting)
bool small_inverse(int n, std::vector<double>& A) {
    std::vector<double> I(n * n, 0.0);
    for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (!(std::fabs(A[piv * n + c]) > 0.0)) return false;
        if (piv != c)
            for (int j = 0; j < n; ++j) {
                std::swap(A[c * n + j], A[piv * n + j]);
                std::swap(I[c * n + j], I[piv * n + j]);
            }
        double p = A[c * n + c];
        for (int j = 0; j < n; ++j) {
            A[c * n + j] /= p;
            I[c * n + j] /= p;
        }
        for (int r = 0; r < n; ++r)
            if (r != c) {
                double f = A[r * n + c];
                if (f == 0.0) continue;
                for (int j = 0; j < n; ++j) {
                    A[r * n + j] -= f * A[c * n + j];
                    I[r * n + j] -= f * I[c * n + j];
                }
            }
    }
    A = I;
    return true;
}

// Conjugate gradients with block-Jacobi preconditioning (blocks = one soft
// vertex (3) or one affine body (12)), relative residual tolerance rtol.
bool cg_solve(int n, const std::vector<Trip>& T, const std::vector<double>& b, const std::vector<int>& blk_off,
              const std::vector<int>& blk_n, double rtol, std::vector<double>& x) {
    // CSR
    std::vector<Trip> S = T;
    std::sort(S.begin(), S.end(), [](const Trip& a, const Trip& c) { return a.i != c.i ? a.i < c.i : a.j < c.j; });
    std::vector<int> rp(n + 1, 0), ci;
    std::vector<double> vv;
    for (size_t k = 0; k < S.size();) {
        size_t e = k;
        double s = 0.0;
        while (e < S.size() && S[e].i == S[k].i && S[e].j == S[k].j) s += S[e++].v;
        ci.push_back(S[k].j);
        vv.push_back(s);
        rp[S[k].i + 1]++;
        k = e;
    }
    for (int i = 0; i < n; ++i) rp[i + 1] += rp[i];
    auto spmv = [&](const std::vector<double>& in, std::vector<double>& o) {
        ORC_PARALLEL_FOR
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int k = rp[i]; k < rp[i + 1]; ++k) s += vv[k] * in[ci[k]];
            o[i] = s;
        }
    };
    // preconditioner blocks
    std::vector<std::vector<double>> inv(blk_off.size());
    for (size_t bi = 0; bi < blk_off.size(); ++bi) {
        int o = blk_off[bi], m = blk_n[bi];
        std::vector<double> A(m * m, 0.0);
        for (int i = 0; i < m; ++i)
            for (int k = rp[o + i]; k < rp[o + i + 1]; ++k)
                if (ci[k] >= o && ci[k] < o + m) A[i * m + (ci[k] - o)] = vv[k];
        if (!small_inverse(m, A)) return false;
        inv[bi] = A;
    }
    auto prec = [&](const std::vector<double>& r, std::vector<double>& z) {
        ORC_PARALLEL_FOR
        for (long bi = 0; bi < (long)blk_off.size(); ++bi) {
            int o = blk_off[bi], m = blk_n[bi];
            for (int i = 0; i < m; ++i) {
                double s = 0.0;
                for (int j = 0; j < m; ++j) s += inv[bi][i * m + j] * r[o + j];
                z[o + i] = s;
            }
        }
    };
    x.assign(n, 0.0);
    std::vector<double> r = b, z(n), p(n), Ap(n);
    double bn = 0.0;
    for (double t : b) bn += t * t;
    bn = std::sqrt(bn);
    if (bn == 0.0) return true;
    prec(r, z);
    p = z;
    double rz = 0.0;
    for (int i = 0; i < n; ++i) rz += r[i] * z[i];
    for (int it = 0; it < 200000; ++it) {
        spmv(p, Ap);
        double pAp = 0.0;
        for (int i = 0; i < n; ++i) pAp += p[i] * Ap[i];
        double a = rz / pAp;
        double rn = 0.0;
        for (int i = 0; i < n; ++i) {
            x[i] += a * p[i];
            r[i] -= a * Ap[i];
            rn += r[i] * r[i];
        }
        if (std::sqrt(rn) <= rtol * bn) return true;
        prec(r, z);
        double rz2 = 0.0;
        for (int i = 0; i < n; ++i) rz2 += r[i] * z[i];
        double beta = rz2 / rz;
        rz = rz2;
        for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    return false;
}

// ===========================================================================
// Energy, gradient and projected Hessian of one environment
// ===========================================================================
struct State {
    std::vector<double> x;  // all soft positions
    std::vector<double> q;  // all affine states (12 per body)
};

void load_dofs(const Scene&, const EnvDofs& D, const std::vector<double>& y, State& st) {
    for (int i : D.verts)
        for (int k = 0; k < 3; ++k) st.x[3 * i + k] = y[D.vert_dof[i] + k];
    for (int a : D.affs)
        for (int k = 0; k < 12; ++k) st.q[12 * a + k] = y[D.aff_dof[a] + k];
}

void store_dofs(const Scene&, const EnvDofs& D, const State& st, std::vector<double>& y) {
    y.assign(D.n, 0.0);
    for (int i : D.verts)
        for (int k = 0; k < 3; ++k) y[D.vert_dof[i] + k] = st.x[3 * i + k];
    for (int a : D.affs)
        for (int k = 0; k < 12; ++k) y[D.aff_dof[a] + k] = st.q[12 * a + k];
}

// deformation gradient F = Ds Dm^-1 (row-major)
void def_grad(const Scene& S, int t, const std::vector<double>& xs, double F[9]) {
    const int* T = &S.tets[4 * t];
    double Ds[9];
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 3; ++r) Ds[3 * r + c] = xs[3 * T[c + 1] + r] - xs[3 * T[0] + r];
    const double* Dm = &S.Dminv[9 * t];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Ds[3 * r + k] * Dm[3 * k + c];
            F[3 * r + c] = s;
        }
}

// dF/dx: B (9 x 12), F_rc depends on x_{v, r} through Dminv
void dFdx(const Scene& S, int t, double B[9][12]) {
    const double* Dm = &S.Dminv[9 * t];
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 12; ++j) B[i][j] = 0.0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            // F_rc = sum_k (x_{k+1,r} - x_{0,r}) Dm_kc
            double s0 = 0.0;
            for (int k = 0; k < 3; ++k) {
                B[3 * r + c][3 * (k + 1) + r] += Dm[3 * k + c];
                s0 += Dm[3 * k + c];
            }
            B[3 * r + c][r] -= s0;
        }
}

struct EvalOpt {
    bool grad, hess;
};

// Total incremental potential of env at state st.  Contact terms use `pairs`
// (all candidate pairs; only those with d < dhat contribute).  Returns +inf
// for an inverted tet or a non-positive distance.
// joint constraint c (12) from the two bodies' q = (p, rows of A):
// c = (A1 B1 - A2 B2 , r x a), r = (A1 y1 + p1) - (A2 y2 + p2), a = A1 d1
template <class T>
void joint_constraint(const Joint& J, const T* q1, const T* q2, T* c) {
    auto A1 = [&](int i, int k) { return q1[3 + 3 * i + k]; };
    auto A2 = [&](int i, int k) { return q2[3 + 3 * i + k]; };
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            T v = (A1(i, 0) * J.B1[j] + A1(i, 1) * J.B1[3 + j]) + A1(i, 2) * J.B1[6 + j];
            v = v - ((A2(i, 0) * J.B2[j] + A2(i, 1) * J.B2[3 + j]) + A2(i, 2) * J.B2[6 + j]);
            c[3 * i + j] = v;
        }
    T r[3], a[3];
    for (int i = 0; i < 3; ++i) {
        T w1 = q1[i] + ((A1(i, 0) * J.y1[0] + A1(i, 1) * J.y1[1]) + A1(i, 2) * J.y1[2]);
        T w2 = q2[i] + ((A2(i, 0) * J.y2[0] + A2(i, 1) * J.y2[1]) + A2(i, 2) * J.y2[2]);
        r[i] = w1 - w2;
        a[i] = (A1(i, 0) * J.d1[0] + A1(i, 1) * J.d1[1]) + A1(i, 2) * J.d1[2];
    }
    c[9] = r[1] * a[2] - r[2] * a[1];
    c[10] = r[2] * a[0] - r[0] * a[2];
    c[11] = r[0] * a[1] - r[1] * a[0];
}

double env_energy(const Scene& S, int env, const EnvDofs& D, const State& st, const std::vector<Pair>& pairs,
                  Sys* Y, EvalOpt opt, int* n_active = nullptr, double* dmin = nullptr) {
    const double h = S.P.dt, h2 = h * h;
    double E = 0.0;
    if (Y) {
        Y->n = D.n;
        Y->g.assign(D.n, 0.0);
        Y->H.clear();
    }
    // soft inertia (Eq. 1)
    for (int i : D.verts) {
        double m = S.mass[i];
        int o = D.vert_dof[i];
        for (int k = 0; k < 3; ++k) {
            double d = st.x[3 * i + k] - S.xhat[3 * i + k];
            E += 0.5 * m * d * d;
            if (Y && opt.grad) Y->g[o + k] += m * d;
            if (Y && opt.hess) Y->H.push_back(Trip{o + k, o + k, m});
        }
        // spring constraint: a potential energy, so scaled by h^2 like the
        // elastic term: h^2 k |x - x_target|^2
        const double ks = S.spring_k.empty() ? 0.0 : S.spring_k[i];
        if (ks > 0.0)
            for (int k = 0; k < 3; ++k) {
                double r = st.x[3 * i + k] - S.spring_x[3 * i + k];
                E += h2 * ks * r * r;
                if (Y && opt.grad) Y->g[o + k] += 2.0 * h2 * ks * r;
                if (Y && opt.hess) Y->H.push_back(Trip{o + k, o + k, 2.0 * h2 * ks});
            }
    }
    // elasticity (Eq. 1, h^2 Phi): per tet of the env, its density psi,
    // x-space gradient gx and PSD-projected Hessian Hx (each tet on its own,
    // in parallel under OpenMP), then summed in tet order
    std::vector<int> etets;
    for (size_t t = 0; t < S.tet_body.size(); ++t)
        if (S.soft[S.bodies[S.tet_body[t]].second].env == env) etets.push_back((int)t);
    const bool tet_der = Y && (opt.grad || opt.hess);
    const size_t ntl = etets.size();
    std::vector<double> tpsi(ntl), tgx(tet_der ? 12 * ntl : 0), tHx(tet_der && opt.hess ? 144 * ntl : 0);
    std::vector<char> tok(ntl, 1);
    ORC_PARALLEL_FOR_DYNAMIC
    for (long l = 0; l < (long)ntl; ++l) {
        const int t = etets[l];
        int sb = S.bodies[S.tet_body[t]].second;
        double F[9];
        def_grad(S, t, st.x, F);
        D2<9> psi;
        if (S.soft[sb].model == 1)
            psi = stvk_psi(F, S.soft[sb].mu_l, S.soft[sb].lam_l);
        else if (S.soft[sb].model == 2) {
            if (!fcr_psi(F, S.soft[sb].mu_l, S.soft[sb].lam_l, psi)) {
                tok[l] = 0;
                continue;
            }
        } else if (!nh_psi(F, S.soft[sb].mu_l, S.soft[sb].lam_l, psi)) {
            tok[l] = 0;
            continue;
        }
        tpsi[l] = psi.v;
        if (!tet_der) continue;
        double w = h2 * S.tvol[t];
        double B[9][12];
        dFdx(S, t, B);
        double* gx = &tgx[12 * l];
        for (int j = 0; j < 12; ++j) {
            gx[j] = 0.0;
            for (int i = 0; i < 9; ++i) gx[j] += B[i][j] * psi.g[i];
        }
        if (!opt.hess) continue;
        double HF[81];
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) HF[9 * i + j] = psi.h[i][j];
        psd_project(9, HF);
        double* Hx = &tHx[144 * l];
        for (int a = 0; a < 12; ++a)
            for (int b = 0; b < 12; ++b) {
                double s = 0.0;
                for (int i = 0; i < 9; ++i)
                    for (int j = 0; j < 9; ++j) s += B[i][a] * HF[9 * i + j] * B[j][b];
                Hx[12 * a + b] = w * s;
            }
    }
    for (size_t l = 0; l < ntl; ++l) {
        if (!tok[l]) return INF;
        const int t = etets[l];
        double w = h2 * S.tvol[t];
        E += w * tpsi[l];
        if (tet_der) {
            const int* T = &S.tets[4 * t];
            const double* gx = &tgx[12 * l];
            const double* Hx = opt.hess ? &tHx[144 * l] : nullptr;
            for (int va = 0; va < 4; ++va) {
                int oa = D.vert_dof[T[va]];
                if (opt.grad)
                    for (int k = 0; k < 3; ++k) Y->g[oa + k] += w * gx[3 * va + k];
                if (opt.hess)
                    for (int vb = 0; vb < 4; ++vb) {
                        int ob = D.vert_dof[T[vb]];
                        add_block(*Y, oa, 3, ob, 3, &Hx[12 * (3 * va) + 3 * vb], 12);
                    }
            }
        }
    }
    // affine inertia and orthogonality (Eq. 2) and kinematic AL (Eq. 13)
    for (int a : D.affs) {
        const Affine& A = S.aff[a];
        const double* q = &st.q[12 * a];
        int o = D.aff_dof[a];
        double dq[12];
        for (int k = 0; k < 12; ++k) dq[k] = q[k] - A.qhat[k];
        double Mdq[12];
        for (int i = 0; i < 12; ++i) {
            double s = 0.0;
            for (int j = 0; j < 12; ++j) s += A.M[12 * i + j] * dq[j];
            Mdq[i] = s;
        }
        for (int i = 0; i < 12; ++i) E += 0.5 * dq[i] * Mdq[i];
        if (Y && opt.grad)
            for (int i = 0; i < 12; ++i) Y->g[o + i] += Mdq[i];
        if (Y && opt.hess) add_block(*Y, o, 12, o, 12, A.M, 12);
        D2<9> ph = ortho(q + 3);
        double w = h2 * A.stiffness * A.vol;
        E += w * ph.v;
        if (Y && opt.grad)
            for (int i = 0; i < 9; ++i) Y->g[o + 3 + i] += w * ph.g[i];
        if (Y && opt.hess) {
            double H9[81];
            for (int i = 0; i < 9; ++i)
                for (int j = 0; j < 9; ++j) H9[9 * i + j] = w * ph.h[i][j];
            psd_project(9, H9);
            add_block(*Y, o + 3, 9, o + 3, 9, H9, 9);
        }
        if (A.mode == 2) {
            double kA = 1e3 * A.m, sm = std::sqrt(A.m);
            for (int i = 0; i < 12; ++i) {
                double d = q[i] - A.qtarget[i];
                E += 0.5 * kA * d * d - sm * A.lamA[i] * d;
                if (Y && opt.grad) Y->g[o + i] += kA * d - sm * A.lamA[i];
                if (Y && opt.hess) Y->H.push_back(Trip{o + i, o + i, kA});
            }
        }
    }
    // prismatic joints: kappa |c|^2 - lambda . c over the free bodies' DOFs
    // (fixed bodies enter as constants); exact Hessian, PSD-projected
    for (const Joint& J : S.joints) {
        if (J.env != env) continue;
        const int o1 = D.aff_dof[J.a1], o2 = D.aff_dof[J.a2];
        D2<24> v1[12], v2[12];
        for (int k = 0; k < 12; ++k) {
            v1[k] = o1 >= 0 ? var<24>(st.q[12 * J.a1 + k], k) : cst<24>(st.q[12 * J.a1 + k]);
            v2[k] = o2 >= 0 ? var<24>(st.q[12 * J.a2 + k], 12 + k) : cst<24>(st.q[12 * J.a2 + k]);
        }
        D2<24> c[12];
        joint_constraint(J, v1, v2, c);
        D2<24> e = cst<24>(0.0);
        for (int m = 0; m < 12; ++m) e = e + (J.kappa * (c[m] * c[m]) + (-J.lam[m]) * c[m]);
        E += e.v;
        if (Y && (opt.grad || opt.hess)) {
            int idx[24], off[24], nf = 0;
            for (int k = 0; k < 12; ++k)
                if (o1 >= 0) {
                    idx[nf] = k;
                    off[nf++] = o1 + k;
                }
            for (int k = 0; k < 12; ++k)
                if (o2 >= 0) {
                    idx[nf] = 12 + k;
                    off[nf++] = o2 + k;
                }
            if (opt.grad)
                for (int a = 0; a < nf; ++a) Y->g[off[a]] += e.g[idx[a]];
            if (opt.hess) {
                std::vector<double> Hf((size_t)nf * nf);
                for (int a = 0; a < nf; ++a)
                    for (int b = 0; b < nf; ++b) Hf[(size_t)a * nf + b] = e.h[idx[a]][idx[b]];
                psd_project(nf, Hf.data());
                for (int a = 0; a < nf; ++a)
                    for (int b = 0; b < nf; ++b) Y->H.push_back(Trip{off[a], off[b], Hf[(size_t)a * nf + b]});
            }
        }
    }
    // barrier (Eq. 4, Eq. 5, coupling Eq. 6-8)
    std::vector<P3> P;
    all_sv_pos(S, st.x, st.q, P);
    double kap = S.kappa[env];
    int nact = 0;
    double dm = INF;
    // per pair: distance, and for an active pair its barrier value, gradient
    // and PSD-projected Hessian (each pair on its own, in parallel under
    // OpenMP); the sums below then run in pair order
    const bool pair_der = Y && (opt.grad || opt.hess);
    const size_t npr = pairs.size();
    std::vector<double> pd(npr), pb(npr), pgl(pair_der ? 12 * npr : 0), pHl(pair_der ? 144 * npr : 0);
    ORC_PARALLEL_FOR_DYNAMIC
    for (long k = 0; k < (long)npr; ++k) {
        const Pair& pr = pairs[k];
        double x12[12];
        stencil(P, pr, x12);
        double d2 = stencil_d2(x12, pr.is_ee);
        if (!(d2 > 0.0)) {
            pd[k] = -1.0;
            continue;
        }
        double d = std::sqrt(d2);
        pd[k] = d;
        if (!(d < S.P.dhat)) continue;
        double epsx = pr.is_ee ? ee_eps_x(S, pr) : 0.0;
        if (!pair_der) {
            double b = barrier(d, S.P.dhat);
            if (pr.is_ee) b *= ee_mollifier_value(x12, epsx);
            pb[k] = b;
            continue;
        }
        D2<12> b;
        pair_barrier(x12, pr.is_ee, S.P.dhat, epsx, b);
        pb[k] = b.v;
        double* gl = &pgl[12 * k];
        double* Hl = &pHl[144 * k];
        for (int i = 0; i < 12; ++i) {
            gl[i] = kap * b.g[i];
            for (int j = 0; j < 12; ++j) Hl[12 * i + j] = kap * b.h[i][j];
        }
        psd_project(12, Hl);  // projected in the 12-dim pair space (Eq. 8)
    }
    for (size_t pi = 0; pi < npr; ++pi) {
        const Pair& pr = pairs[pi];
        const double d = pd[pi];
        if (d < 0.0) return INF;
        dm = std::min(dm, d);
        if (!(d < S.P.dhat)) continue;
        ++nact;
        E += kap * pb[pi];
        if (!pair_der) continue;
        const double* gl = &pgl[12 * pi];
        const double* Hl = &pHl[144 * pi];
        int off[4], nd[4];
        double J[4][3][12];
        for (int k = 0; k < 4; ++k) nd[k] = sv_jac(S, D, pr.s[k], off[k], J[k]);
        for (int ka = 0; ka < 4; ++ka) {
            if (!nd[ka]) continue;
            if (opt.grad)
                for (int c = 0; c < nd[ka]; ++c) {
                    double s = 0.0;
                    for (int i = 0; i < 3; ++i) s += J[ka][i][c] * gl[3 * ka + i];
                    Y->g[off[ka] + c] += s;
                }
            if (opt.hess)
                for (int kb = 0; kb < 4; ++kb) {
                    if (!nd[kb]) continue;
                    double M[144];
                    for (int c = 0; c < nd[ka]; ++c)
                        for (int e = 0; e < nd[kb]; ++e) {
                            double s = 0.0;
                            for (int i = 0; i < 3; ++i)
                                for (int j = 0; j < 3; ++j)
                                    s += J[ka][i][c] * Hl[12 * (3 * ka + i) + 3 * kb + j] * J[kb][j][e];
                            M[12 * c + e] = s;
                        }
                    add_block(*Y, off[ka], nd[ka], off[kb], nd[kb], M, 12);
                }
        }
    }
    if (n_active) *n_active = nact;
    if (dmin) *dmin = dm;
    // lagged friction (Eq. 9, Eq. 10)
    const double eh = S.P.eps_v * h;
    std::vector<P3> Pt;
    {
        // x^t positions of surface vertices
        std::vector<double> qt(S.aff.size() * 12);
        for (size_t a = 0; a < S.aff.size(); ++a)
            for (int k = 0; k < 12; ++k) qt[12 * a + k] = S.aff[a].qt[k];
        all_sv_pos(S, S.xt, qt, Pt);
    }
    for (const Lagged& L : S.lagged[env]) {
        P3 Dl{0, 0, 0};
        for (int k = 0; k < 4; ++k) Dl = add(Dl, mul(L.w[k], sub(P[L.s[k]], Pt[L.s[k]])));
        P3 n = p3(L.n);
        P3 u = sub(Dl, mul(dot(n, Dl), n));  // tangential part (I - n n^T) Delta
        double y = std::sqrt(dot(u, u));
        double c = L.mu * L.lam;
        E += c * f0(y, eh);
        if (!(Y && (opt.grad || opt.hess))) continue;
        // gradient and Hessian with respect to Delta (3)
        double gD[3], HD[9];
        double T[9];
        double nv[3] = {n.x, n.y, n.z}, uv[3] = {u.x, u.y, u.z};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) T[3 * i + j] = (i == j ? 1.0 : 0.0) - nv[i] * nv[j];
        double a1, a2;  // H = c (a1 T + a2 u u^T)
        if (y >= eh) {
            a1 = 1.0 / y;
            a2 = -1.0 / (y * y * y);
        } else {
            a1 = 2.0 / eh - y / (eh * eh);
            a2 = (y > 0.0) ? -1.0 / (eh * eh * y) : 0.0;
        }
        double f1y = (y >= eh) ? 1.0 / y : (2.0 / eh - y / (eh * eh));  // f1(y)/y
        for (int i = 0; i < 3; ++i) gD[i] = c * f1y * uv[i];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) HD[3 * i + j] = c * (a1 * T[3 * i + j] + a2 * uv[i] * uv[j]);
        int off[4], nd[4];
        double J[4][3][12];
        for (int k = 0; k < 4; ++k) nd[k] = sv_jac(S, D, L.s[k], off[k], J[k]);
        for (int ka = 0; ka < 4; ++ka) {
            if (!nd[ka] || L.w[ka] == 0.0) continue;
            if (opt.grad)
                for (int cc = 0; cc < nd[ka]; ++cc) {
                    double s = 0.0;
                    for (int i = 0; i < 3; ++i) s += J[ka][i][cc] * gD[i];
                    Y->g[off[ka] + cc] += L.w[ka] * s;
                }
            if (opt.hess)
                for (int kb = 0; kb < 4; ++kb) {
                    if (!nd[kb] || L.w[kb] == 0.0) continue;
                    double M[144];
                    for (int c1 = 0; c1 < nd[ka]; ++c1)
                        for (int c2 = 0; c2 < nd[kb]; ++c2) {
                            double s = 0.0;
                            for (int i = 0; i < 3; ++i)
                                for (int j = 0; j < 3; ++j) s += J[ka][i][c1] * HD[3 * i + j] * J[kb][j][c2];
                            M[12 * c1 + c2] = L.w[ka] * L.w[kb] * s;
                        }
                    add_block(*Y, off[ka], nd[ka], off[kb], nd[kb], M, 12);
                }
        }
    }
    return E;
}

// ===========================================================================
// Additive CCD (ACCD) for one pair: fraction t in (0, t_c] of the step p that
// is safe.  Steps follow the additive CCD of Li, Kaufman, Jiang (2021) with
// thickness 0: remove the mean displacement, bound the closing speed by the
// sum of the largest displacement norms on each side, and advance by
// (1 - s) d / l_p first and 0.9 d / l_p afterwards until the distance falls
// below s times its initial value.
// ===========================================================================
double accd(const double* x12in, const double* p12in, bool is_ee, double s, double tc, int max_iter,
            int* iters = nullptr) {
    double x[12], p[12];
    for (int i = 0; i < 12; ++i) {
        x[i] = x12in[i];
        p[i] = p12in[i];
    }
    double mean[3] = {0, 0, 0};
    for (int k = 0; k < 4; ++k)
        for (int i = 0; i < 3; ++i) mean[i] += 0.25 * p[3 * k + i];
    for (int k = 0; k < 4; ++k)
        for (int i = 0; i < 3; ++i) p[3 * k + i] -= mean[i];
    double nrm[4];
    for (int k = 0; k < 4; ++k)
        nrm[k] = std::sqrt(p[3 * k] * p[3 * k] + p[3 * k + 1] * p[3 * k + 1] + p[3 * k + 2] * p[3 * k + 2]);
    double lp = is_ee ? std::max(nrm[0], nrm[1]) + std::max(nrm[2], nrm[3])
                      : nrm[0] + std::max(nrm[1], std::max(nrm[2], nrm[3]));
    if (iters) *iters = 0;
    if (lp == 0.0) return tc;
    double d = std::sqrt(stencil_d2(x, is_ee));
    double g = s * d;
    double t = 0.0;
    double tl = (1.0 - s) * d / lp;
    for (int it = 0; it < max_iter; ++it) {
        for (int i = 0; i < 12; ++i) x[i] += tl * p[i];
        d = std::sqrt(stencil_d2(x, is_ee));
        if (iters) *iters = it + 1;
        if (t > 0.0 && d < g) break;
        t += tl;
        if (t > tc) return tc;
        tl = 0.9 * d / lp;
    }
    return t;
}

// min(1, ACCD bound of every swept pair) for the motion P0 -> P1 (s = 0.1,
// t_c = 1): each pair's bound on its own (in parallel under OpenMP), then
// the minimum in pair order
double swept_accd_min(const std::vector<P3>& P0, const std::vector<P3>& P1, const std::vector<Pair>& swept) {
    std::vector<double> tb(swept.size());
    ORC_PARALLEL_FOR_DYNAMIC
    for (long k = 0; k < (long)swept.size(); ++k) {
        const Pair& pr = swept[k];
        double x12[12], e12[12], p12[12];
        stencil(P0, pr, x12);
        stencil(P1, pr, e12);
        for (int i = 0; i < 12; ++i) p12[i] = e12[i] - x12[i];
        tb[k] = accd(x12, p12, pr.is_ee, 0.1, 1.0, 10000);
    }
    double alpha = 1.0;
    for (double t : tb) alpha = std::min(alpha, t);
    return alpha;
}

// ===========================================================================
// Time stepping
// ===========================================================================
double bbox_diag_all(const Scene& S) {
    double lo[3] = {INF, INF, INF}, hi[3] = {-INF, -INF, -INF};
    std::vector<double> qs(S.aff.size() * 12);
    for (size_t a = 0; a < S.aff.size(); ++a)
        for (int k = 0; k < 12; ++k) qs[12 * a + k] = S.aff[a].q[k];
    for (size_t s = 0; s < S.sv.size(); ++s) {
        P3 p = sv_pos(S, (int)s, S.x, qs);
        double c[3] = {p.x, p.y, p.z};
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], c[k]);
            hi[k] = std::max(hi[k], c[k]);
        }
    }
    // interior soft vertices count too
    for (size_t i = 0; i < S.x.size() / 3; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], S.x[3 * i + k]);
            hi[k] = std::max(hi[k], S.x[3 * i + k]);
        }
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) d2 += (hi[k] - lo[k]) * (hi[k] - lo[k]);
    return std::sqrt(d2);
}

void get_state(const Scene& S, State& st) {
    st.x = S.x;
    st.q.assign(S.aff.size() * 12, 0.0);
    for (size_t a = 0; a < S.aff.size(); ++a)
        for (int k = 0; k < 12; ++k) st.q[12 * a + k] = S.aff[a].q[k];
}

// Newton step norm: max abs component over soft vertices and affine mesh
// vertices (J p_b)
double step_inf_norm(const Scene& S, const EnvDofs& D, const std::vector<double>& p) {
    double m = 0.0;
    for (int i : D.verts)
        for (int k = 0; k < 3; ++k) m = std::max(m, std::fabs(p[D.vert_dof[i] + k]));
    for (int a : D.affs) {
        const Affine& A = S.aff[a];
        const double* pb = &p[D.aff_dof[a]];
        for (size_t v = 0; v < A.V.size() / 3; ++v) {
            const double* x0 = &A.V[3 * v];
            for (int i = 0; i < 3; ++i) {
                double s = pb[i] + pb[3 + 3 * i] * x0[0] + pb[3 + 3 * i + 1] * x0[1] + pb[3 + 3 * i + 2] * x0[2];
                m = std::max(m, std::fabs(s));
            }
        }
    }
    return m;
}

enum Status { OK = 0, E_INVALID = 1, E_NEWTON = 6, E_LS = 7, E_LIN = 8, E_NONFINITE = 9 };

// Normal-force magnitude, weights and normal of every active pair at x^t
void lag_friction(Scene& S, int env) {
    State st;
    get_state(S, st);
    std::vector<P3> P;
    all_sv_pos(S, st.x, st.q, P);
    std::vector<Pair> pairs;
    candidate_pairs(S, env, P, nullptr, pairs);
    S.lagged[env].clear();
    for (const Pair& pr : pairs) {
        double x12[12];
        stencil(P, pr, x12);
        Cand c = pr.is_ee ? ee_closest(x12) : pt_closest(x12);
        double d = std::sqrt(c.d2);
        if (!(d < S.P.dhat)) continue;
        double e = pr.is_ee ? ee_mollifier_value(x12, ee_eps_x(S, pr)) : 1.0;
        Lagged L;
        L.is_ee = pr.is_ee;
        for (int k = 0; k < 4; ++k) {
            L.s[k] = pr.s[k];
            L.w[k] = 0.0;
        }
        for (int k = 0; k < c.na; ++k) L.w[c.a[k]] += c.w[k];
        P3 dv{0, 0, 0};
        for (int k = 0; k < 4; ++k) dv = add(dv, mul(L.w[k], P[pr.s[k]]));
        double dl = std::sqrt(dot(dv, dv));
        L.n[0] = dv.x / dl;
        L.n[1] = dv.y / dl;
        L.n[2] = dv.z / dl;
        L.lam = S.kappa[env] * e * std::fabs(barrier_d1(d, S.P.dhat));
        int b0 = S.sv[pr.s[0]].body, b1 = S.sv[pr.s[pr.is_ee ? 2 : 1]].body;
        L.mu = std::min(body_mu(S, b0), body_mu(S, b1));
        S.lagged[env].push_back(L);
    }
}

void init_kappa(Scene& S, int env) {
    // kappa_min from the mean soft lumped mass, else mean affine mass / 8
    double sm = 0.0;
    int cnt = 0;
    for (size_t i = 0; i < S.mass.size(); ++i)
        if (body_env(S, S.vert_body[i]) == env) {
            sm += S.mass[i];
            ++cnt;
        }
    double mbar;
    if (cnt > 0)
        mbar = sm / cnt;
    else {
        double s2 = 0.0;
        int c2 = 0;
        for (const Affine& A : S.aff)
            if (A.env == env && A.mode == 0) {
                s2 += A.m / 8.0;
                ++c2;
            }
        mbar = c2 ? s2 / c2 : 1.0;
    }
    S.kappa_min[env] = 1e3 * mbar;
    if (S.P.kappa > 0.0) {
        S.kappa[env] = S.P.kappa;
        return;
    }
    // gradient balance at x^t: kappa = -gE . gB / |gB|^2
    EnvDofs D = env_dofs(S, env);
    State st;
    get_state(S, st);
    std::vector<P3> P;
    all_sv_pos(S, st.x, st.q, P);
    std::vector<Pair> pairs;
    candidate_pairs(S, env, P, nullptr, pairs);
    double keep = S.kappa[env];
    auto lag = S.lagged[env];
    S.lagged[env].clear();
    Sys Yall, Yb;
    S.kappa[env] = 1.0;
    env_energy(S, env, D, st, pairs, &Yall, EvalOpt{true, false});
    std::vector<Pair> none;
    Sys Ye;
    env_energy(S, env, D, st, none, &Ye, EvalOpt{true, false});
    S.kappa[env] = keep;
    S.lagged[env] = lag;
    double gg = 0.0, bb = 0.0;
    for (int i = 0; i < D.n; ++i) {
        double gb = Yall.g[i] - Ye.g[i];
        gg += Ye.g[i] * gb;
        bb += gb * gb;
    }
    double k = S.kappa_min[env];
    if (bb > 0.0) k = std::min(std::max(-gg / bb, S.kappa_min[env]), 100.0 * S.kappa_min[env]);
    S.kappa[env] = k;
}

double env_dmin(const Scene& S, int env) {
    State st;
    get_state(S, st);
    std::vector<P3> P;
    all_sv_pos(S, st.x, st.q, P);
    std::vector<Pair> pairs;
    candidate_pairs(S, env, P, nullptr, pairs);
    double dm = INF;
    for (const Pair& pr : pairs) {
        double x12[12];
        stencil(P, pr, x12);
        double d = std::sqrt(stencil_d2(x12, pr.is_ee));
        if (d < S.P.dhat) dm = std::min(dm, d);
    }
    return dm;
}

void commit_state(Scene& S, const State& st) {
    S.x = st.x;
    for (size_t a = 0; a < S.aff.size(); ++a)
        for (int k = 0; k < 12; ++k) S.aff[a].q[k] = st.q[12 * a + k];
}

// The Newton system H p = rhs of an env: `which` 0 as the stepper solves it
// (dense Cholesky up to 2,500 DOF, else CG with block-Jacobi blocks of one
// soft vertex (3) or one affine body (12) to relative residual 1e-12),
// 1 dense Cholesky, 2 that CG.
bool newton_solve(const EnvDofs& D, const Sys& Y, const std::vector<double>& rhs, std::vector<double>& p, int which) {
    if (which == 1 || (which == 0 && D.n <= 2500)) return dense_solve(D.n, Y.H, rhs, p);
    std::vector<int> bo, bn;
    for (int i : D.verts) {
        bo.push_back(D.vert_dof[i]);
        bn.push_back(3);
    }
    for (int a : D.affs) {
        bo.push_back(D.aff_dof[a]);
        bn.push_back(12);
    }
    return cg_solve(D.n, Y.H, rhs, bo, bn, 1e-12, p);
}

int newton_env(Scene& S, int env, double tol, StepStats& ss) {
    EnvDofs D = env_dofs(S, env);
    State st;
    get_state(S, st);
    std::vector<double> y;
    store_dofs(S, D, st, y);
    for (int it = 0; it < S.P.max_newton; ++it) {
        load_dofs(S, D, y, st);
        std::vector<P3> P;
        all_sv_pos(S, st.x, st.q, P);
        std::vector<Pair> pairs;
        candidate_pairs(S, env, P, nullptr, pairs);
        Sys Y;
        int nact = 0;
        double E0 = env_energy(S, env, D, st, pairs, &Y, EvalOpt{true, true}, &nact);
        if (!std::isfinite(E0)) return E_NONFINITE;
        S.energy_log.push_back(E0);
        ss.n_active = nact;
        std::vector<double> rhs(D.n), p;
        for (int i = 0; i < D.n; ++i) rhs[i] = -Y.g[i];
        if (!newton_solve(D, Y, rhs, p, 0)) return E_LIN;
        if (step_inf_norm(S, D, p) <= tol) {
            ss.energy = E0;
            commit_state(S, st);
            return OK;
        }
        ss.newton_iters += 1;
        // CCD bound over swept candidates
        State s1 = st;
        std::vector<double> y1(D.n);
        for (int i = 0; i < D.n; ++i) y1[i] = y[i] + p[i];
        load_dofs(S, D, y1, s1);
        std::vector<P3> P1;
        all_sv_pos(S, s1.x, s1.q, P1);
        std::vector<Pair> swept;
        candidate_pairs(S, env, P, &P1, swept);
        double alpha = swept_accd_min(P, P1, swept);
        // backtracking line search on the energy over the swept candidates
        double Eprev = env_energy(S, env, D, st, swept, nullptr, EvalOpt{false, false});
        bool acc = false;
        for (int k = 0; k <= 60; ++k) {
            for (int i = 0; i < D.n; ++i) y1[i] = y[i] + alpha * p[i];
            load_dofs(S, D, y1, s1);
            double E1 = env_energy(S, env, D, s1, swept, nullptr, EvalOpt{false, false});
            if (E1 <= Eprev) {
                acc = true;
                break;
            }
            alpha *= 0.5;
            ss.ls_halvings += 1;
        }
        if (!acc) return E_LS;
        y = y1;
    }
    return E_NEWTON;
}

// Predictor (Eq. 1, Eq. 2, Eq. 3): x^ = x^t + h v^t + h^2 M^-1 f_e for the
// soft vertices, q^ = q^t + h qdot^t + h^2 M_b^-1 f_e for the affine bodies,
// with f_e the gravity load (integral of rho J^T g over the body).
void predict(Scene& S, int env) {
    const double h = S.P.dt;
    EnvDofs D = env_dofs(S, env);
    for (int i : D.verts) {
        double m = S.mass[i];
        for (int k = 0; k < 3; ++k) {
            S.xt[3 * i + k] = S.x[3 * i + k];
            double fe = m * S.P.g[k];
            S.xhat[3 * i + k] = S.x[3 * i + k] + h * S.v[3 * i + k] + h * h * fe / m;
        }
    }
    for (size_t a = 0; a < S.aff.size(); ++a) {
        Affine& A = S.aff[a];
        if (A.env != env) continue;
        for (int k = 0; k < 12; ++k) A.qt[k] = A.q[k];
        if (A.mode == 1) {
            for (int k = 0; k < 12; ++k) A.qhat[k] = A.q[k];
            continue;
        }
        double c[3] = {A.M[3], A.M[4], A.M[5]};  // integral rho x0
        double fe[12];
        for (int i = 0; i < 3; ++i) fe[i] = A.m * S.P.g[i];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) fe[3 + 3 * i + k] = S.P.g[i] * c[k];
        std::vector<double> Mi(A.M, A.M + 144);
        small_inverse(12, Mi);
        for (int i = 0; i < 12; ++i) {
            double s = 0.0;
            for (int j = 0; j < 12; ++j) s += Mi[12 * i + j] * fe[j];
            A.qhat[i] = A.q[i] + h * A.qd[i] + h * h * s;
        }
    }
}

// Warm start: propose x^0 = x^t + alpha Delta with Delta = h v^t (soft) and
// h qdot^t (non-fixed affine), alpha the ACCD bound over the swept candidates
// of x^t -> x^t + Delta; keep the proposal only if it does not raise the
// energy, else start from x^t.
void warm_start(Scene& S, int env, StepStats& ss) {
    const double h = S.P.dt;
    EnvDofs D = env_dofs(S, env);
    State st;
    get_state(S, st);
    std::vector<double> y0, y1(D.n), dl(D.n, 0.0);
    store_dofs(S, D, st, y0);
    bool any = false;
    for (int i : D.verts)
        for (int k = 0; k < 3; ++k) {
            dl[D.vert_dof[i] + k] = h * S.v[3 * i + k];
            any |= dl[D.vert_dof[i] + k] != 0.0;
        }
    for (int a : D.affs)
        for (int k = 0; k < 12; ++k) {
            dl[D.aff_dof[a] + k] = h * S.aff[a].qd[k];
            any |= dl[D.aff_dof[a] + k] != 0.0;
        }
    if (!any) return;
    for (int i = 0; i < D.n; ++i) y1[i] = y0[i] + dl[i];
    State s1 = st;
    load_dofs(S, D, y1, s1);
    std::vector<P3> P0, P1;
    all_sv_pos(S, st.x, st.q, P0);
    all_sv_pos(S, s1.x, s1.q, P1);
    std::vector<Pair> swept;
    candidate_pairs(S, env, P0, &P1, swept);
    double alpha = swept_accd_min(P0, P1, swept);
    for (int i = 0; i < D.n; ++i) y1[i] = y0[i] + alpha * dl[i];
    load_dofs(S, D, y1, s1);
    double E0 = env_energy(S, env, D, st, swept, nullptr, EvalOpt{false, false});
    double E1 = env_energy(S, env, D, s1, swept, nullptr, EvalOpt{false, false});
    if (E1 <= E0) {
        commit_state(S, s1);
        ss.warm_accepted = 1;
    }
}

int step_env(Scene& S, int env, StepStats& ss) {
    const double h = S.P.dt;
    EnvDofs D = env_dofs(S, env);
    // the augmented-Lagrangian iteration of Eq. 13 starts from the linear
    // extrapolation of the last two steps' converged multipliers (a reading:
    // the paper does not say where it starts)
    if (S.P.al_extrapolate)
        for (Affine& A : S.aff) {
            if (A.env != env || A.mode != 2) continue;
            for (int k = 0; k < 12; ++k) {
                const double l = A.lamA[k];
                A.lamA[k] = 2.0 * l - A.lamA_prev[k];
                A.lamA_prev[k] = l;
            }
        }
    predict(S, env);
    if (!S.kappa_init[env]) {
        init_kappa(S, env);
        S.dmin_last[env] = env_dmin(S, env);
        S.kappa_init[env] = 1;
    }
    lag_friction(S, env);
    warm_start(S, env, ss);
    double tol = S.P.tol_rel * S.diag[env] * h;
    int status = OK;
    int rounds = 0;
    for (;;) {
        status = newton_env(S, env, tol, ss);
        if (status != OK) break;
        // kinematic AL multiplier update
        bool any = false;
        for (size_t a = 0; a < S.aff.size(); ++a) {
            Affine& A = S.aff[a];
            if (A.env != env || A.mode != 2) continue;
            double m = 0.0;
            for (int k = 0; k < 12; ++k) m = std::max(m, std::fabs(A.q[k] - A.qtarget[k]));
            if (m > tol) any = true;
        }
        // prismatic joints: rotation part within tol_rel h, slide part
        // within the step tolerance
        std::vector<std::array<double, 12>> jc(S.joints.size());
        for (size_t j = 0; j < S.joints.size(); ++j) {
            const Joint& J = S.joints[j];
            if (J.env != env) continue;
            joint_constraint(J, S.aff[J.a1].q, S.aff[J.a2].q, jc[j].data());
            for (int m = 0; m < 12; ++m)
                if (std::fabs(jc[j][m]) > (m < 9 ? S.P.tol_rel * h : tol)) any = true;
        }
        if (!any || rounds >= S.P.max_al_rounds) break;
        ++rounds;
        for (size_t a = 0; a < S.aff.size(); ++a) {
            Affine& A = S.aff[a];
            if (A.env != env || A.mode != 2) continue;
            double kA = 1e3 * A.m, sm = std::sqrt(A.m);
            for (int k = 0; k < 12; ++k) A.lamA[k] -= kA * (A.q[k] - A.qtarget[k]) / sm;
        }
        for (size_t j = 0; j < S.joints.size(); ++j) {
            Joint& J = S.joints[j];
            if (J.env != env) continue;
            for (int m = 0; m < 12; ++m) J.lam[m] -= 2.0 * J.kappa * jc[j][m];
        }
    }
    ss.al_rounds = rounds;
    if (status != OK) return status;
    // with the extrapolation, the step ends with one more multiplier update
    // from the accepted state (no new solve), so that the values the next
    // step extrapolates from carry no part of the deviation the tolerance let
    // through
    if (S.P.al_extrapolate)
        for (Affine& A : S.aff) {
            if (A.env != env || A.mode != 2) continue;
            const double kA = 1e3 * A.m, sm = std::sqrt(A.m);
            for (int k = 0; k < 12; ++k) A.lamA[k] -= kA * (A.q[k] - A.qtarget[k]) / sm;
        }
    // velocities (Eq. 11)
    for (int i : D.verts)
        for (int k = 0; k < 3; ++k) S.v[3 * i + k] = (S.x[3 * i + k] - S.xt[3 * i + k]) / h;
    for (size_t a = 0; a < S.aff.size(); ++a) {
        Affine& A = S.aff[a];
        if (A.env != env || A.mode == 1) continue;
        for (int k = 0; k < 12; ++k) A.qd[k] = (A.q[k] - A.qt[k]) / h;
    }
    // kappa adaptation
    double dm = env_dmin(S, env);
    if (S.P.kappa <= 0.0 && dm < 0.1 * S.P.dhat && dm < S.dmin_last[env])
        S.kappa[env] = std::min(2.0 * S.kappa[env], 1e4 * S.kappa_min[env]);
    S.dmin_last[env] = dm;
    ss.dmin = dm;
    ss.kappa = S.kappa[env];
    return OK;
}

}  // namespace

// ===========================================================================
// C interface for the tests (ctypes)
// ===========================================================================
extern "C" {

// dparams: dt, dhat, kappa, eps_v, tol_rel, gx, gy, gz, pcg_rel_tol
// iparams: max_newton, max_al_rounds, n_envs, al_extrapolate
void* orc_create(const double* dp, const int* ip) {
    Scene* S = new Scene();
    S->P.dt = dp[0];
    S->P.dhat = dp[1];
    S->P.kappa = dp[2];
    S->P.eps_v = dp[3];
    S->P.tol_rel = dp[4];
    S->P.g[0] = dp[5];
    S->P.g[1] = dp[6];
    S->P.g[2] = dp[7];
    S->P.pcg_rel_tol = dp[8];
    S->P.max_newton = ip[0];
    S->P.max_al_rounds = ip[1];
    S->n_envs = ip[2];
    S->P.al_extrapolate = ip[3];
    return S;
}

void orc_destroy(void* s) { delete (Scene*)s; }

int orc_add_tet_body(void* s, int env, const double* X, long nv, const int* tets, long nt, const double* x0,
                     const double* v0, double E, double nu, double rho, double mu) {
    Scene& S = *(Scene*)s;
    if (S.finalized || env < 0 || env >= S.n_envs) return -E_INVALID;
    int body = (int)S.bodies.size();
    SoftBody B;
    B.env = env;
    B.v0 = (int)(S.X.size() / 3);
    B.nv = (int)nv;
    B.t0 = (int)(S.tets.size() / 4);
    B.nt = (int)nt;
    B.mu_l = E / (2.0 * (1.0 + nu));
    B.lam_l = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    B.mu = mu;
    B.rho = rho;
    for (long i = 0; i < 3 * nv; ++i) {
        S.X.push_back(X[i]);
        S.x.push_back(x0 ? x0[i] : X[i]);
        S.v.push_back(v0 ? v0[i] : 0.0);
    }
    for (long i = 0; i < nv; ++i) S.vert_body.push_back(body);
    for (long t = 0; t < nt; ++t) {
        for (int k = 0; k < 4; ++k) S.tets.push_back(B.v0 + tets[4 * t + k]);
        S.tet_body.push_back(body);
    }
    S.soft.push_back(B);
    S.bodies.push_back({0, (int)S.soft.size() - 1});
    return body;
}

int orc_add_affine_body(void* s, int env, const double* V, long nv, const int* F, long nf, const double* q0,
                        const double* qd0, double rho, double stiffness, double mu, int mode) {
    Scene& S = *(Scene*)s;
    if (S.finalized || env < 0 || env >= S.n_envs) return -E_INVALID;
    Affine A;
    A.env = env;
    A.mode = mode;
    A.V.assign(V, V + 3 * nv);
    A.F.assign(F, F + 3 * nf);
    A.rho = rho;
    A.stiffness = stiffness;
    A.mu = mu;
    for (int k = 0; k < 12; ++k) {
        A.q[k] = q0[k];
        A.qd[k] = qd0 ? qd0[k] : 0.0;
        A.qtarget[k] = q0[k];
        A.lamA[k] = 0.0;
        A.lamA_prev[k] = 0.0;
    }
    // mass matrix M_b = integral rho J^T J over the body (Eq. 2) via the
    // divergence theorem: tetrahedra (0, a, b, c) over the closed surface
    double m0 = 0.0, m1[3] = {0, 0, 0}, m2[9] = {0};
    for (long f = 0; f < nf; ++f) {
        const double* a = V + 3 * F[3 * f];
        const double* b = V + 3 * F[3 * f + 1];
        const double* c = V + 3 * F[3 * f + 2];
        double vol = (a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                      a[2] * (b[0] * c[1] - b[1] * c[0])) / 6.0;
        m0 += vol;
        double sm[3];
        for (int i = 0; i < 3; ++i) {
            sm[i] = a[i] + b[i] + c[i];
            m1[i] += vol * sm[i] / 4.0;
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                m2[3 * i + j] += vol / 20.0 * (a[i] * a[j] + b[i] * b[j] + c[i] * c[j] + sm[i] * sm[j]);
    }
    A.vol = m0;
    A.m = rho * m0;
    for (int i = 0; i < 144; ++i) A.M[i] = 0.0;
    // ordering (p, a1, a2, a3): x_i = p_i + a_i . x0
    for (int i = 0; i < 3; ++i) {
        A.M[12 * i + i] = A.m;
        for (int k = 0; k < 3; ++k) {
            A.M[12 * i + 3 + 3 * i + k] = rho * m1[k];
            A.M[12 * (3 + 3 * i + k) + i] = rho * m1[k];
        }
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) A.M[12 * (3 + 3 * i + k) + 3 + 3 * i + l] = rho * m2[3 * k + l];
    }
    int body = (int)S.bodies.size();
    S.aff.push_back(A);
    S.bodies.push_back({1, (int)S.aff.size() - 1});
    return body;
}

// prismatic joint between two affine bodies (axis in world coordinates at the
// initial state; kappa <= 0: 1e3 x the mean of the two masses)
int orc_add_prismatic_joint(void* s, int body1, int body2, const double* axis, double kappa) {
    Scene& S = *(Scene*)s;
    const int nb = (int)S.bodies.size();
    if (S.finalized || body1 < 0 || body1 >= nb || body2 < 0 || body2 >= nb || body1 == body2 ||
        S.bodies[body1].first != 1 || S.bodies[body2].first != 1)
        return -E_INVALID;
    Joint J;
    J.a1 = S.bodies[body1].second;
    J.a2 = S.bodies[body2].second;
    const Affine &A1 = S.aff[J.a1], &A2 = S.aff[J.a2];
    if (A1.env != A2.env) return -E_INVALID;
    J.env = A1.env;
    J.kappa = kappa > 0.0 ? kappa : 1e3 * 0.5 * (A1.m + A2.m);
    auto inv = [](const double* M, double* I) {
        double C[9] = {M[4] * M[8] - M[5] * M[7], M[5] * M[6] - M[3] * M[8], M[3] * M[7] - M[4] * M[6],
                       M[2] * M[7] - M[1] * M[8], M[0] * M[8] - M[2] * M[6], M[1] * M[6] - M[0] * M[7],
                       M[1] * M[5] - M[2] * M[4], M[2] * M[3] - M[0] * M[5], M[0] * M[4] - M[1] * M[3]};
        double d = M[0] * C[0] + M[1] * C[1] + M[2] * C[2];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) I[3 * i + j] = C[3 * j + i] / d;
        return d;
    };
    if (!(inv(A1.q + 3, J.B1) > 0.0) || !(inv(A2.q + 3, J.B2) > 0.0)) return -E_INVALID;
    // body 1's centre of mass (rest frame: first moment over mass) in the world
    double w0[3];
    for (int i = 0; i < 3; ++i) {
        w0[i] = A1.q[i];
        for (int k = 0; k < 3; ++k) w0[i] += A1.q[3 + 3 * i + k] * A1.M[3 + k] / A1.m;
    }
    double n = std::sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
    if (!(n > 0.0)) return -E_INVALID;
    for (int i = 0; i < 3; ++i) {
        J.y1[i] = J.y2[i] = J.d1[i] = 0.0;
        for (int k = 0; k < 3; ++k) {
            J.y1[i] += J.B1[3 * i + k] * (w0[k] - A1.q[k]);
            J.y2[i] += J.B2[3 * i + k] * (w0[k] - A2.q[k]);
            J.d1[i] += J.B1[3 * i + k] * axis[k] / n;
        }
    }
    for (int m = 0; m < 12; ++m) J.lam[m] = 0.0;
    S.joints.push_back(J);
    return (int)S.joints.size() - 1;
}

// the 12 constraint values of joint j at the current state
int orc_joint_constraint(void* s, int j, double* c) {
    Scene& S = *(Scene*)s;
    if (j < 0 || j >= (int)S.joints.size()) return -E_INVALID;
    const Joint& J = S.joints[j];
    joint_constraint(J, S.aff[J.a1].q, S.aff[J.a2].q, c);
    return 0;
}

// material of a soft body: 0 Neo-Hookean, 1 St. Venant-Kirchhoff, 2 fixed corotated
int orc_set_material(void* s, int body, int model) {
    Scene& S = *(Scene*)s;
    if (S.finalized || body < 0 || body >= (int)S.bodies.size() || S.bodies[body].first != 0 || model < 0 ||
        model > 2)
        return -E_INVALID;
    S.soft[S.bodies[body].second].model = model;
    return 0;
}

// springs of a soft body (body-local vertices), replacing the body's springs
int orc_set_springs(void* s, int body, const int* verts, long n, const double* targets, double k) {
    Scene& S = *(Scene*)s;
    if (body < 0 || body >= (int)S.bodies.size() || S.bodies[body].first != 0 || n < 0 || !(k >= 0.0))
        return -E_INVALID;
    const SoftBody& B = S.soft[S.bodies[body].second];
    const size_t nvt = S.X.size() / 3;
    if (S.spring_k.size() < nvt) {
        S.spring_k.resize(nvt, 0.0);
        S.spring_x.resize(3 * nvt, 0.0);
    }
    for (int i = 0; i < B.nv; ++i) S.spring_k[B.v0 + i] = 0.0;
    for (long i = 0; i < n; ++i) {
        if (verts[i] < 0 || verts[i] >= B.nv) return -E_INVALID;
        const int g = B.v0 + verts[i];
        S.spring_k[g] = k;
        for (int j = 0; j < 3; ++j) S.spring_x[3 * g + j] = targets[3 * i + j];
    }
    return 0;
}

int orc_finalize(void* s) {
    Scene& S = *(Scene*)s;
    if (S.finalized) return -E_INVALID;
    size_t nvt = S.X.size() / 3;
    S.mass.assign(nvt, 0.0);
    S.xt = S.x;
    S.xhat = S.x;
    size_t nt = S.tets.size() / 4;
    S.Dminv.assign(9 * nt, 0.0);
    S.tvol.assign(nt, 0.0);
    for (size_t t = 0; t < nt; ++t) {
        const int* T = &S.tets[4 * t];
        double Dm[9];
        for (int c = 0; c < 3; ++c)
            for (int r = 0; r < 3; ++r) Dm[3 * r + c] = S.X[3 * T[c + 1] + r] - S.X[3 * T[0] + r];
        double det = Dm[0] * (Dm[4] * Dm[8] - Dm[5] * Dm[7]) - Dm[1] * (Dm[3] * Dm[8] - Dm[5] * Dm[6]) +
                     Dm[2] * (Dm[3] * Dm[7] - Dm[4] * Dm[6]);
        if (!(det > 0.0)) {
            S.err = "inverted rest tet";
            return -E_INVALID;
        }
        std::vector<double> inv(Dm, Dm + 9);
        if (!small_inverse(3, inv)) {
            S.err = "singular rest tet";
            return -E_INVALID;
        }
        for (int k = 0; k < 9; ++k) S.Dminv[9 * t + k] = inv[k];
        S.tvol[t] = det / 6.0;
        int sb = S.bodies[S.tet_body[t]].second;
        for (int k = 0; k < 4; ++k) S.mass[T[k]] += S.soft[sb].rho * S.tvol[t] / 4.0;
    }
    // soft surface: faces that belong to exactly one tet, outward-oriented
    std::map<std::tuple<int, int, int>, std::vector<int>> faces;  // sorted key -> oriented face
    std::map<std::tuple<int, int, int>, int> count;
    static const int FL[4][3] = {{0, 2, 1}, {0, 1, 3}, {0, 3, 2}, {1, 2, 3}};
    for (size_t t = 0; t < nt; ++t) {
        const int* T = &S.tets[4 * t];
        for (int f = 0; f < 4; ++f) {
            int a = T[FL[f][0]], b = T[FL[f][1]], c = T[FL[f][2]];
            int k[3] = {a, b, c};
            std::sort(k, k + 3);
            auto key = std::make_tuple(k[0], k[1], k[2]);
            count[key] += 1;
            faces[key] = {a, b, c};
        }
    }
    std::map<int, int> soft_sv;  // global soft vertex -> surface vertex
    std::vector<std::vector<int>> stris;
    for (auto& kv : count)
        if (kv.second == 1) stris.push_back(faces[kv.first]);
    // order surface triangles by body then by key (map order) for determinism
    for (auto& f : stris)
        for (int v : f)
            if (!soft_sv.count(v)) soft_sv[v] = 0;
    for (auto& kv : soft_sv) {
        kv.second = (int)S.sv.size();
        S.sv.push_back(SV{S.vert_body[kv.first], 0, kv.first});
    }
    std::map<std::pair<int, int>, int> edge_set;
    auto add_tri = [&](int a, int b, int c) {
        S.tris.push_back(a);
        S.tris.push_back(b);
        S.tris.push_back(c);
        int e[3][2] = {{a, b}, {b, c}, {c, a}};
        for (auto& ed : e) {
            auto key = std::make_pair(std::min(ed[0], ed[1]), std::max(ed[0], ed[1]));
            if (!edge_set.count(key)) {
                edge_set[key] = 1;
                S.edges.push_back(key.first);
                S.edges.push_back(key.second);
            }
        }
    };
    for (auto& f : stris) add_tri(soft_sv[f[0]], soft_sv[f[1]], soft_sv[f[2]]);
    // affine surfaces: every mesh vertex is a surface vertex
    for (size_t a = 0; a < S.aff.size(); ++a) {
        Affine& A = S.aff[a];
        int body = -1;
        for (size_t b = 0; b < S.bodies.size(); ++b)
            if (S.bodies[b].first == 1 && S.bodies[b].second == (int)a) body = (int)b;
        A.sv0 = (int)S.sv.size();
        for (size_t v = 0; v < A.V.size() / 3; ++v) S.sv.push_back(SV{body, 1, (int)v});
        for (size_t f = 0; f < A.F.size() / 3; ++f)
            add_tri(A.sv0 + A.F[3 * f], A.sv0 + A.F[3 * f + 1], A.sv0 + A.F[3 * f + 2]);
    }
    // per-env quantities
    S.kappa.assign(S.n_envs, S.P.kappa > 0 ? S.P.kappa : 0.0);
    S.kappa_min.assign(S.n_envs, 0.0);
    S.kappa_init.assign(S.n_envs, 0);
    S.dmin_last.assign(S.n_envs, INF);
    S.lagged.assign(S.n_envs, {});
    double dg = bbox_diag_all(S);
    S.diag.assign(S.n_envs, dg);
    // each env uses the bbox diagonal of its own bodies
    for (int e = 0; e < S.n_envs; ++e) {
        double lo[3] = {INF, INF, INF}, hi[3] = {-INF, -INF, -INF};
        std::vector<double> qs(S.aff.size() * 12);
        for (size_t a = 0; a < S.aff.size(); ++a)
            for (int k = 0; k < 12; ++k) qs[12 * a + k] = S.aff[a].q[k];
        bool any = false;
        for (size_t s = 0; s < S.sv.size(); ++s) {
            if (body_env(S, S.sv[s].body) != e) continue;
            P3 p = sv_pos(S, (int)s, S.x, qs);
            double c[3] = {p.x, p.y, p.z};
            for (int k = 0; k < 3; ++k) {
                lo[k] = std::min(lo[k], c[k]);
                hi[k] = std::max(hi[k], c[k]);
            }
            any = true;
        }
        if (any) {
            double d2 = 0.0;
            for (int k = 0; k < 3; ++k) d2 += (hi[k] - lo[k]) * (hi[k] - lo[k]);
            S.diag[e] = std::sqrt(d2);
        }
    }
    S.finalized = true;
    return 0;
}

int orc_set_kinematic_target(void* s, int body, const double* q) {
    Scene& S = *(Scene*)s;
    if (body < 0 || body >= (int)S.bodies.size() || S.bodies[body].first != 1) return -E_INVALID;
    for (int k = 0; k < 12; ++k) S.aff[S.bodies[body].second].qtarget[k] = q[k];
    return 0;
}

// One or more time steps.  stats: 8 doubles per step per env (StepStats).
int orc_step(void* s, int n, double* stats) {
    Scene& S = *(Scene*)s;
    if (!S.finalized) return -E_INVALID;
    for (int it = 0; it < n; ++it)
        for (int e = 0; e < S.n_envs; ++e) {
            StepStats ss{0, 0, 0, 0, 0, 0, 0, 0, 0};
            // keep the last completed step on failure
            std::vector<double> x0 = S.x, v0 = S.v;
            std::vector<Affine> a0 = S.aff;
            int st = step_env(S, e, ss);
            ss.status = st;
            if (stats) {
                double* o = stats + 8 * ((size_t)it * S.n_envs + e);
                o[0] = ss.newton_iters; o[1] = ss.ls_halvings; o[2] = ss.al_rounds; o[3] = ss.n_active;
                o[4] = ss.dmin; o[5] = ss.energy; o[6] = ss.kappa; o[7] = ss.status;
            }
            if (st != OK) {
                S.x = x0;
                S.v = v0;
                S.aff = a0;
                return -st;
            }
        }
    return 0;
}

// tet body: x then v (nv x 3 each); affine body: q then qdot (12 each)
long orc_get_state(void* s, int body, double* out, long cap) {
    Scene& S = *(Scene*)s;
    if (body < 0 || body >= (int)S.bodies.size()) return -E_INVALID;
    auto bk = S.bodies[body];
    if (bk.first == 0) {
        const SoftBody& B = S.soft[bk.second];
        long n = 6L * B.nv;
        if (cap < n) return -E_INVALID;
        for (long i = 0; i < 3L * B.nv; ++i) {
            out[i] = S.x[3L * B.v0 + i];
            out[3L * B.nv + i] = S.v[3L * B.v0 + i];
        }
        return n;
    }
    const Affine& A = S.aff[bk.second];
    if (cap < 24) return -E_INVALID;
    for (int k = 0; k < 12; ++k) {
        out[k] = A.q[k];
        out[12 + k] = A.qd[k];
    }
    return 24;
}

int orc_set_state(void* s, int body, const double* in, long n) {
    Scene& S = *(Scene*)s;
    if (body < 0 || body >= (int)S.bodies.size()) return -E_INVALID;
    auto bk = S.bodies[body];
    if (bk.first == 0) {
        const SoftBody& B = S.soft[bk.second];
        if (n != 6L * B.nv) return -E_INVALID;
        for (long i = 0; i < 3L * B.nv; ++i) {
            S.x[3L * B.v0 + i] = in[i];
            S.v[3L * B.v0 + i] = in[3L * B.nv + i];
        }
        return 0;
    }
    Affine& A = S.aff[bk.second];
    if (n != 24) return -E_INVALID;
    for (int k = 0; k < 12; ++k) {
        A.q[k] = in[k];
        A.qd[k] = in[12 + k];
    }
    return 0;
}

double orc_kappa(void* s, int env) { return ((Scene*)s)->kappa[env]; }
// energies of all Newton iterates since the last call (then cleared)
long orc_energy_log(void* s, double* out, long cap) {
    Scene& S = *(Scene*)s;
    long n = (long)S.energy_log.size();
    for (long i = 0; i < n && i < cap; ++i) out[i] = S.energy_log[i];
    S.energy_log.clear();
    return n;
}
double orc_diag(void* s, int env) { return ((Scene*)s)->diag[env]; }
double orc_kappa_min(void* s, int env) { return ((Scene*)s)->kappa_min[env]; }
void orc_set_kappa(void* s, int env, double k, double kmin) {
    Scene& S = *(Scene*)s;
    S.kappa[env] = k;
    S.kappa_min[env] = kmin;
    S.kappa_init[env] = 1;
}
int orc_counts(void* s, long* out) {
    Scene& S = *(Scene*)s;
    out[0] = (long)S.sv.size();
    out[1] = (long)S.edges.size() / 2;
    out[2] = (long)S.tris.size() / 3;
    out[3] = (long)S.x.size() / 3;
    out[4] = (long)S.tets.size() / 4;
    return 0;
}
// surface topology: sv (body, affine, idx) triples, edges, tris
int orc_surface(void* s, int* sv3, int* edges, int* tris) {
    Scene& S = *(Scene*)s;
    for (size_t i = 0; i < S.sv.size(); ++i) {
        sv3[3 * i] = S.sv[i].body;
        sv3[3 * i + 1] = S.sv[i].affine;
        sv3[3 * i + 2] = S.sv[i].idx;
    }
    std::copy(S.edges.begin(), S.edges.end(), edges);
    std::copy(S.tris.begin(), S.tris.end(), tris);
    return 0;
}
int orc_lumped_mass(void* s, double* out) {
    Scene& S = *(Scene*)s;
    std::copy(S.mass.begin(), S.mass.end(), out);
    return 0;
}
int orc_affine_mass(void* s, int body, double* M144, double* mv) {
    Scene& S = *(Scene*)s;
    if (S.bodies[body].first != 1) return -E_INVALID;
    const Affine& A = S.aff[S.bodies[body].second];
    std::copy(A.M, A.M + 144, M144);
    mv[0] = A.m;
    mv[1] = A.vol;
    return 0;
}

// ---------------------------------------------------------------------------
// Env-level evaluation for derivative checks.  Sets up x^ and the lagged
// friction from the current state exactly as a step would (without changing
// the state), then evaluates E, gradient and the dense projected Hessian at
// the env DOF vector y (nullable outputs).
// ---------------------------------------------------------------------------
int orc_env_ndof(void* s, int env) { return env_dofs(*(Scene*)s, env).n; }

int orc_env_dofs(void* s, int env, double* y) {
    Scene& S = *(Scene*)s;
    EnvDofs D = env_dofs(S, env);
    State st;
    get_state(S, st);
    std::vector<double> v;
    store_dofs(S, D, st, v);
    std::copy(v.begin(), v.end(), y);
    return D.n;
}

// Prepare x^t, x^ (and kappa, lagged friction) for env as the start of a step.
int orc_prepare(void* s, int env, int with_friction) {
    Scene& S = *(Scene*)s;
    predict(S, env);
    if (!S.kappa_init[env]) {
        init_kappa(S, env);
        S.dmin_last[env] = env_dmin(S, env);
        S.kappa_init[env] = 1;
    }
    if (with_friction)
        lag_friction(S, env);
    else
        S.lagged[env].clear();
    return 0;
}

double orc_env_eval(void* s, int env, const double* y, double* g, double* H, int* n_active) {
    Scene& S = *(Scene*)s;
    EnvDofs D = env_dofs(S, env);
    State st;
    get_state(S, st);
    std::vector<double> yy(y, y + D.n);
    load_dofs(S, D, yy, st);
    std::vector<P3> P;
    all_sv_pos(S, st.x, st.q, P);
    std::vector<Pair> pairs;
    candidate_pairs(S, env, P, nullptr, pairs);
    Sys Y;
    double E = env_energy(S, env, D, st, pairs, (g || H) ? &Y : nullptr, EvalOpt{g != nullptr, H != nullptr},
                          n_active);
    if (g)
        for (int i = 0; i < D.n; ++i) g[i] = Y.g[i];
    if (H) {
        std::fill(H, H + (size_t)D.n * D.n, 0.0);
        for (const Trip& t : Y.H) H[(size_t)t.i * D.n + t.j] += t.v;
    }
    return E;
}

// Newton system of env at DOF vector y (as orc_env_eval assembles it) solved
// for p = -H^-1 g with newton_solve's `which` (0 the stepper's choice, 1 dense
// Cholesky, 2 CG); p: n doubles.  Returns 0, or -1 if the solve failed.
int orc_newton_system_solve(void* s, int env, const double* y, int which, double* p) {
    Scene& S = *(Scene*)s;
    EnvDofs D = env_dofs(S, env);
    State st;
    get_state(S, st);
    std::vector<double> yy(y, y + D.n);
    load_dofs(S, D, yy, st);
    std::vector<P3> P;
    all_sv_pos(S, st.x, st.q, P);
    std::vector<Pair> pairs;
    candidate_pairs(S, env, P, nullptr, pairs);
    Sys Y;
    env_energy(S, env, D, st, pairs, &Y, EvalOpt{true, true});
    std::vector<double> rhs(D.n), out;
    for (int i = 0; i < D.n; ++i) rhs[i] = -Y.g[i];
    if (!newton_solve(D, Y, rhs, out, which)) return -1;
    std::copy(out.begin(), out.end(), p);
    return 0;
}

// Contact force sensing (paper section on contact force sensing): per body
// b, out[3 b .. 3 b + 2] = (1 / h^2) sum over the body's surface vertices v
// of dB/dx_v, B = kappa e b(d) summed over the pairs with d < dhat at the
// current state (all pairs by brute force).  Returns 0.
int orc_contact_forces(void* s, double* out) {
    Scene& S = *(Scene*)s;
    State st;
    get_state(S, st);
    std::vector<P3> P;
    all_sv_pos(S, st.x, st.q, P);
    std::fill(out, out + 3 * S.bodies.size(), 0.0);
    const double h2 = S.P.dt * S.P.dt;
    for (int env = 0; env < S.n_envs; ++env) {
        std::vector<Pair> pairs;
        candidate_pairs(S, env, P, nullptr, pairs);
        for (const Pair& pr : pairs) {
            double x12[12];
            stencil(P, pr, x12);
            D2<12> b;
            if (!pair_barrier(x12, pr.is_ee, S.P.dhat, pr.is_ee ? ee_eps_x(S, pr) : 0.0, b)) continue;
            for (int k = 0; k < 4; ++k) {
                const int body = S.sv[pr.s[k]].body;
                for (int i = 0; i < 3; ++i) out[3 * body + i] += S.kappa[env] * b.g[3 * k + i] / h2;
            }
        }
    }
    return 0;
}

// OpenMP threads of the parallel loops (results do not depend on it); the
// library starts with 1.  n <= 0 only reads.  Returns the count in use (1
// without OpenMP).
int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) g_orc_threads = n;
    return g_orc_threads;
#else
    (void)n;
    return 1;
#endif
}

// ---------------------------------------------------------------------------
// Local functions for the pins
// ---------------------------------------------------------------------------
// Squared distance of a PT (is_ee = 0) or EE stencil with its kind, weights,
// gradient and Hessian of d^2 (nullable).
double orc_stencil_d2(const double* x12, int is_ee, int* kind, double* w4, double* g12, double* H144) {
    Cand c = is_ee ? ee_closest(x12) : pt_closest(x12);
    if (kind) *kind = c.kind;
    if (w4) {
        for (int k = 0; k < 4; ++k) w4[k] = 0.0;
        for (int k = 0; k < c.na; ++k) w4[c.a[k]] += c.w[k];
    }
    if (g12 || H144) {
        D2<12> d = cand_d2(x12, c, is_ee);
        for (int i = 0; i < 12; ++i) {
            if (g12) g12[i] = d.g[i];
            if (H144)
                for (int j = 0; j < 12; ++j) H144[12 * i + j] = d.h[i][j];
        }
    }
    return c.d2;
}

// Barrier of one stencil with gradient and PSD-projected (project != 0) or
// exact Hessian; eps_x only for EE.  Returns 0 for inactive pairs.
double orc_pair_barrier(const double* x12, int is_ee, double dhat, double eps_x, int project, double* g12,
                        double* H144) {
    D2<12> b;
    if (!pair_barrier(x12, is_ee != 0, dhat, eps_x, b)) {
        if (g12) std::fill(g12, g12 + 12, 0.0);
        if (H144) std::fill(H144, H144 + 144, 0.0);
        return 0.0;
    }
    if (g12)
        for (int i = 0; i < 12; ++i) g12[i] = b.g[i];
    if (H144) {
        for (int i = 0; i < 12; ++i)
            for (int j = 0; j < 12; ++j) H144[12 * i + j] = b.h[i][j];
        if (project) psd_project(12, H144);
    }
    return b.v;
}

double orc_barrier_scalar(double d, double dhat) { return barrier(d, dhat); }
double orc_f0(double y, double eh) { return f0(y, eh); }
double orc_f1(double y, double eh) { return f1(y, eh); }

// Neo-Hookean Psi(F) with F-space gradient (9) and Hessian (81, projected if asked)
double orc_nh(const double* F9, double mu, double lam, int project, double* g9, double* H81) {
    D2<9> p;
    if (!nh_psi(F9, mu, lam, p)) return INF;
    if (g9)
        for (int i = 0; i < 9; ++i) g9[i] = p.g[i];
    if (H81) {
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) H81[9 * i + j] = p.h[i][j];
        if (project) psd_project(9, H81);
    }
    return p.v;
}

// St. Venant-Kirchhoff Psi(F) with F-space gradient (9) and Hessian (81,
// projected if asked)
double orc_stvk(const double* F9, double mu, double lam, int project, double* g9, double* H81) {
    D2<9> p = stvk_psi(F9, mu, lam);
    if (g9)
        for (int i = 0; i < 9; ++i) g9[i] = p.g[i];
    if (H81) {
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) H81[9 * i + j] = p.h[i][j];
        if (project) psd_project(9, H81);
    }
    return p.v;
}

// fixed-corotated Psi(F) (+inf for J <= 0) with gradient and Hessian
double orc_fcr(const double* F9, double mu, double lam, int project, double* g9, double* H81) {
    D2<9> p;
    if (!fcr_psi(F9, mu, lam, p)) return INF;
    if (g9)
        for (int i = 0; i < 9; ++i) g9[i] = p.g[i];
    if (H81) {
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) H81[9 * i + j] = p.h[i][j];
        if (project) psd_project(9, H81);
    }
    return p.v;
}

double orc_ortho(const double* A9, double* g9, double* H81) {
    D2<9> p = ortho(A9);
    if (g9)
        for (int i = 0; i < 9; ++i) g9[i] = p.g[i];
    if (H81)
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) H81[9 * i + j] = p.h[i][j];
    return p.v;
}

double orc_accd(const double* x12, const double* p12, int is_ee, double s, double tc, int* iters) {
    return accd(x12, p12, is_ee != 0, s, tc, 10000, iters);
}

int orc_eigvals(int n, const double* A, double* ev) {
    std::vector<double> M(A, A + n * n), e, V;
    jacobi_eigen(n, M, e, V);
    std::copy(e.begin(), e.end(), ev);
    return 0;
}

// Brute-force candidate pairs of a raw surface (no scene): all valid PT and EE
// pairs whose AABBs, inflated by infl, overlap (swept when pos1 is given).
// sv_body / body_class / body_env describe the filters; out arrays sized by
// the caller (cap pairs each); returns the counts in n_out[2].
int orc_brute_pairs(long nsv, const double* pos0, const double* pos1, const int* sv_body, long nb,
                    const int* b_class, const int* b_env, long ne, const int* edges, long nt, const int* tris,
                    double infl, long cap, int* pt_out, int* ee_out, long* n_out) {
    Scene S;
    S.bodies.resize(nb);
    // fake bodies with the requested classes and envs
    for (long b = 0; b < nb; ++b) {
        if (b_class[b] == 0) {
            SoftBody B{};
            B.env = b_env[b];
            S.soft.push_back(B);
            S.bodies[b] = {0, (int)S.soft.size() - 1};
        } else {
            Affine A{};
            A.env = b_env[b];
            A.mode = b_class[b] == 1 ? 0 : (b_class[b] == 2 ? 1 : 2);
            S.aff.push_back(A);
            S.bodies[b] = {1, (int)S.aff.size() - 1};
        }
    }
    S.sv.resize(nsv);
    for (long s = 0; s < nsv; ++s) S.sv[s] = SV{sv_body[s], b_class[sv_body[s]] != 0, (int)s};
    S.edges.assign(edges, edges + 2 * ne);
    S.tris.assign(tris, tris + 3 * nt);
    S.P.dhat = 2.0 * infl;
    std::vector<P3> P0(nsv), P1(nsv);
    for (long s = 0; s < nsv; ++s) {
        P0[s] = p3(pos0 + 3 * s);
        if (pos1) P1[s] = p3(pos1 + 3 * s);
    }
    long npt = 0, nee = 0;
    int n_envs = 0;
    for (long b = 0; b < nb; ++b) n_envs = std::max(n_envs, b_env[b] + 1);
    for (int e = 0; e < n_envs; ++e) {
        std::vector<Pair> out;
        candidate_pairs(S, e, P0, pos1 ? &P1 : nullptr, out);
        for (const Pair& p : out) {
            if (p.is_ee) {
                if (nee < cap)
                    for (int k = 0; k < 4; ++k) ee_out[4 * nee + k] = p.s[k];
                ++nee;
            } else {
                if (npt < cap)
                    for (int k = 0; k < 4; ++k) pt_out[4 * npt + k] = p.s[k];
                ++npt;
            }
        }
    }
    n_out[0] = npt;
    n_out[1] = nee;
    return 0;
}

}  // extern "C"
