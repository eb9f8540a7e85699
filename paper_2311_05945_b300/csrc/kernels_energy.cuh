// Energy terms of the incremental potential (Eq. 1-5, Eq. 9-10, Eq. 13):
// per-element gradients and PSD-projected Hessians written to staging
// buffers, and energy-only evaluations reduced per environment.
#pragma once
#include "barrier_coop.cuh"
#include "distance.cuh"
#include "scene.cuh"

namespace zema {

// Energy terms reduced per environment (partial sums per block chunk).
enum ETerm { ET_INERTIA = 0, ET_ELASTIC = 1, ET_AFFINE = 2, ET_BARRIER = 3, ET_FRICTION = 4, ET_JOINT = 5, ET_COUNT = 6 };

// Sum over i in [lo, hi) of f(i) by block (chunk = blockIdx.x) of env
// blockIdx.y, fixed order; thread 0 writes the block's partial.
template <class F>
__device__ __forceinline__ void chunk_sum(int lo, int hi, F f, double* out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = lo + blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += gridDim.x * blockDim.x) s += f(i);
    double t = block_sum<kRedThreads>(s, sh);
    if (threadIdx.x == 0) *out = t;
}

__device__ __forceinline__ double* part_slot(double* part, int term, int n_envs, int env) {
    return part + ((size_t)term * n_envs + env) * kChunks + blockIdx.x;
}

// ---------------------------------------------------------------------------
// Neo-Hookean density Psi(F) = mu/2 (tr F^T F - 3) - mu ln J + lam/2 (ln J)^2
// (the material used for the soft solids), its first Piola stress P and the
// F-space Hessian d2Psi/dF2 = mu I + h'' g g^T + h' d2J/dF2 with g = dJ/dF
// (cofactor matrix) and h(J) = -mu ln J + lam/2 (ln J)^2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int lc(int a, int b, int c) { return (a - b) * (b - c) * (c - a) / 2; }

__device__ inline bool nh_eval(const double* F, double mu, double lam, double& psi, double* P, SMat<9>* H) {
    double g[9];
    g[0] = F[4] * F[8] - F[5] * F[7];
    g[1] = F[5] * F[6] - F[3] * F[8];
    g[2] = F[3] * F[7] - F[4] * F[6];
    g[3] = F[2] * F[7] - F[1] * F[8];
    g[4] = F[0] * F[8] - F[2] * F[6];
    g[5] = F[1] * F[6] - F[0] * F[7];
    g[6] = F[1] * F[5] - F[2] * F[4];
    g[7] = F[2] * F[3] - F[0] * F[5];
    g[8] = F[0] * F[4] - F[1] * F[3];
    double J = F[0] * g[0] + F[1] * g[1] + F[2] * g[2];
    if (!(J > 0.0)) return false;
    double lj = log(J);
    double tr = 0.0;
    for (int i = 0; i < 9; ++i) tr += F[i] * F[i];
    psi = 0.5 * mu * (tr - 3.0) - mu * lj + 0.5 * lam * lj * lj;
    double h1 = (lam * lj - mu) / J;
    double h2 = (lam * (1.0 - lj) + mu) / (J * J);
    if (P)
        for (int i = 0; i < 9; ++i) P[i] = mu * F[i] + h1 * g[i];
    if (H) {
        SMat<9>& M = *H;
        for (int a = 0; a < 9; ++a)
            for (int b = 0; b < 9; ++b) M(a, b) = h2 * g[a] * g[b] + (a == b ? mu : 0.0);
        // d2J / dF_ij dF_kl = eps_ikm eps_jln F_mn (nonzero only for i != k, j != l)
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
                if (i == k) continue;
                int m = 3 - i - k;
                int eik = lc(i, k, m);
                for (int j = 0; j < 3; ++j)
                    for (int l = 0; l < 3; ++l) {
                        if (j == l) continue;
                        int n = 3 - j - l;
                        M(3 * i + j, 3 * k + l) += h1 * eik * lc(j, l, n) * F[3 * m + n];
                    }
            }
    }
    return true;
}

// ---------------------------------------------------------------------------
// PSD projection of the Neo-Hookean F-space Hessian from its analytic
// eigensystem (isotropic energies: Smith, de Goes, Kim 2019).  With the SVD
// F = U diag(s) V^T (det U = det V = 1, s > 0 since J > 0) and
// Psi_i = dPsi/ds_i = mu s_i - c / s_i, c = mu - lam ln J:
//   flip  (u_i v_j^T + u_j v_i^T)/sqrt2 : (Psi_i - Psi_j)/(s_i - s_j) = mu + c/(s_i s_j)
//   twist (u_i v_j^T - u_j v_i^T)/sqrt2 : (Psi_i + Psi_j)/(s_i + s_j) = mu - c/(s_i s_j)
//   scaling sum_i a_i u_i v_i^T, a an eigenvector of the 3x3
//     A_ii = mu + (c + lam)/s_i^2, A_ij = lam/(s_i s_j)
// H = sum_k max(lambda_k, 0) q_k q_k^T over the nine orthonormal q_k.
// ---------------------------------------------------------------------------
// symmetric 3x3 eigen-decomposition by cyclic Jacobi (a overwritten;
// eigenvalues on its diagonal, eigenvectors in the columns of Q)
template <class T>
__device__ inline void sym3_eigen(T a[3][3], T Q[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Q[i][j] = i == j ? T(1) : T(0);
    for (int sweep = 0; sweep < 12; ++sweep) {
        T off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        T dg = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (off <= Eps<T>::off2 * T(0.01) * dg) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                T apq = a[p][q];
                if (apq == T(0)) continue;
                T tau = (a[q][q] - a[p][p]) / (T(2) * apq);
                T t = copysign(T(1), tau) / (fabs(tau) + sqrt(T(1) + tau * tau));
                T cs = rsqrt(T(1) + t * t), sn = t * cs;
                for (int k = 0; k < 3; ++k) {
                    T akp = a[k][p], akq = a[k][q];
                    a[k][p] = cs * akp - sn * akq;
                    a[k][q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    T apk = a[p][k], aqk = a[q][k];
                    a[p][k] = cs * apk - sn * aqk;
                    a[q][k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    T qkp = Q[k][p], qkq = Q[k][q];
                    Q[k][p] = cs * qkp - sn * qkq;
                    Q[k][q] = sn * qkp + cs * qkq;
                }
            }
    }
}

// projected H_F into M (9x9, row-major vec(F) indices 3r + c), computed in T;
// false if J <= 0
template <class T>
__device__ inline bool nh_hessian_projected(const double* Fd, double mu_d, double lam_d, SMat<9, T> M) {
    double Jd = Fd[0] * (Fd[4] * Fd[8] - Fd[5] * Fd[7]) - Fd[1] * (Fd[3] * Fd[8] - Fd[5] * Fd[6]) +
                Fd[2] * (Fd[3] * Fd[7] - Fd[4] * Fd[6]);
    if (!(Jd > 0.0)) return false;
    T F[9];
    for (int i = 0; i < 9; ++i) F[i] = (T)Fd[i];
    const T mu = (T)mu_d, lam = (T)lam_d;
    // V, s from F^T F
    T C[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C[i][j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
    sym3_eigen<T>(C, V);
    T detV = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) - V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
             V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
    if (detV < T(0))
        for (int k = 0; k < 3; ++k) V[k][2] = -V[k][2];
    T sg[3], U[3][3];
    for (int i = 0; i < 3; ++i) sg[i] = sqrt(fmax(C[i][i], T(0)));
    for (int i = 0; i < 3; ++i)
        for (int r = 0; r < 3; ++r) U[r][i] = (F[3 * r] * V[0][i] + F[3 * r + 1] * V[1][i] + F[3 * r + 2] * V[2][i]) / sg[i];
    T c = (T)(mu_d - lam_d * log(Jd));
    for (int a = 0; a < 9; ++a)
        for (int b = 0; b < 9; ++b) M(a, b) = T(0);
    const T is2 = T(0.70710678118654752440);
    // twist and flip modes of each pair (i, j)
    for (int i = 0; i < 2; ++i)
        for (int j = i + 1; j < 3; ++j) {
            T ss = sg[i] * sg[j];
            T lf = fmax(mu + c / ss, T(0)), lt = fmax(mu - c / ss, T(0));
            if (lf == T(0) && lt == T(0)) continue;
            T qf[9], qt[9];
            for (int r = 0; r < 3; ++r)
                for (int cc = 0; cc < 3; ++cc) {
                    T x = U[r][i] * V[cc][j], y = U[r][j] * V[cc][i];
                    qf[3 * r + cc] = is2 * (x + y);
                    qt[3 * r + cc] = is2 * (x - y);
                }
            for (int a = 0; a < 9; ++a)
                for (int b = 0; b < 9; ++b) M(a, b) += lf * qf[a] * qf[b] + lt * qt[a] * qt[b];
        }
    // scaling modes
    T A[3][3], Qa[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A[i][j] = i == j ? mu + (c + lam) / (sg[i] * sg[i]) : lam / (sg[i] * sg[j]);
    sym3_eigen<T>(A, Qa);
    for (int k = 0; k < 3; ++k) {
        T lk = fmax(A[k][k], T(0));
        if (lk == T(0)) continue;
        T q[9];
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc)
                q[3 * r + cc] = Qa[0][k] * U[r][0] * V[cc][0] + Qa[1][k] * U[r][1] * V[cc][1] + Qa[2][k] * U[r][2] * V[cc][2];
        for (int a = 0; a < 9; ++a)
            for (int b = 0; b < 9; ++b) M(a, b) += lk * q[a] * q[b];
    }
    return true;
}

// D[v][c]: derivative of F_rc with respect to x_{v, r} (rows of Dm^-1; v = 0
// gets minus their sum)
__device__ __forceinline__ void dF_coef(const double* Dm, double D[4][3]) {
    for (int c = 0; c < 3; ++c) {
        D[1][c] = Dm[c];
        D[2][c] = Dm[3 + c];
        D[3][c] = Dm[6 + c];
        D[0][c] = -(D[1][c] + D[2][c] + D[3][c]);
    }
}

// ---------------------------------------------------------------------------
// St. Venant-Kirchhoff density (a material choice of the paper's soft
// solids): E = (F^T F - I) / 2, Psi = mu E:E + lam/2 tr(E)^2, first Piola
// stress P = F S with S = 2 mu E + lam tr(E) I.  Defined for every F
// (no barrier against inversion).
// ---------------------------------------------------------------------------
__device__ inline void stvk_eval(const double* F, double mu, double lam, double& psi, double* P) {
    double E[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double c = 0.0;
            for (int k = 0; k < 3; ++k) c += F[3 * k + i] * F[3 * k + j];
            E[3 * i + j] = 0.5 * (c - (i == j ? 1.0 : 0.0));
        }
    const double tr = E[0] + E[4] + E[8];
    double ee = 0.0;
    for (int i = 0; i < 9; ++i) ee += E[i] * E[i];
    psi = mu * ee + 0.5 * lam * tr * tr;
    if (!P) return;
    double S[9];
    for (int i = 0; i < 9; ++i) S[i] = 2.0 * mu * E[i] + (i % 4 == 0 ? lam * tr : 0.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
            for (int k = 0; k < 3; ++k) v += F[3 * i + k] * S[3 * k + j];
            P[3 * i + j] = v;
        }
}

// F-space Hessian of StVK, column (a, b) = dP for dF = e_a e_b^T:
//   dP = dF S + F dS, dS = 2 mu dE + lam tr(dE) I,
//   dE_ij = (delta_ib F_aj + F_ai delta_jb) / 2, tr(dE) = F_ab;
// then projected onto the PSD cone (cyclic Jacobi: the StVK Hessian has no
// simple closed eigensystem).  W is 81 values of scratch.
template <class T>
__device__ inline void stvk_hessian_projected(const double* F, double mu, double lam, SMat<9, T> H, T* W) {
    double E[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double c = 0.0;
            for (int k = 0; k < 3; ++k) c += F[3 * k + i] * F[3 * k + j];
            E[3 * i + j] = 0.5 * (c - (i == j ? 1.0 : 0.0));
        }
    const double tr = E[0] + E[4] + E[8];
    double S[9];
    for (int i = 0; i < 9; ++i) S[i] = 2.0 * mu * E[i] + (i % 4 == 0 ? lam * tr : 0.0);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double dS[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    const double dE = 0.5 * ((i == b ? F[3 * a + j] : 0.0) + (j == b ? F[3 * a + i] : 0.0));
                    dS[3 * i + j] = 2.0 * mu * dE + (i == j ? lam * F[3 * a + b] : 0.0);
                }
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double v = i == a ? S[3 * b + j] : 0.0;
                    for (int k = 0; k < 3; ++k) v += F[3 * i + k] * dS[3 * k + j];
                    H(3 * i + j, 3 * a + b) = (T)v;
                }
        }
    psd_project<9, T>(H, SMat<9, T>{W, 1});
}

// ---------------------------------------------------------------------------
// Fixed-corotated density (a material choice of the paper's soft solids):
// Psi = mu |F - R|^2 + lam/2 (J - 1)^2 with R the rotation of the polar
// decomposition F = R S, here for J > 0 only (J <= 0: +inf, as for
// Neo-Hookean, so R is always a proper rotation).
// P = 2 mu (F - R) + lam (J - 1) cof(F).
// ---------------------------------------------------------------------------
__device__ inline void cof3(const double* A, double* C) {
    C[0] = A[4] * A[8] - A[5] * A[7];
    C[1] = A[5] * A[6] - A[3] * A[8];
    C[2] = A[3] * A[7] - A[4] * A[6];
    C[3] = A[2] * A[7] - A[1] * A[8];
    C[4] = A[0] * A[8] - A[2] * A[6];
    C[5] = A[1] * A[6] - A[0] * A[7];
    C[6] = A[1] * A[5] - A[2] * A[4];
    C[7] = A[2] * A[3] - A[0] * A[5];
    C[8] = A[0] * A[4] - A[1] * A[3];
}

// rotation of the polar decomposition by Newton's iteration
// R <- (R + R^-T) / 2 from R = F (quadratic convergence for det F > 0)
__device__ inline bool polar_rotation(const double* F, double* R) {
    for (int i = 0; i < 9; ++i) R[i] = F[i];
    for (int it = 0; it < 60; ++it) {
        double C[9];
        cof3(R, C);
        const double det = R[0] * C[0] + R[1] * C[1] + R[2] * C[2];
        if (!(det > 0.0)) return false;
        double diff = 0.0;
        for (int i = 0; i < 9; ++i) {
            const double r = 0.5 * (R[i] + C[i] / det);
            diff = fmax(diff, fabs(r - R[i]));
            R[i] = r;
        }
        if (diff < 1e-15) break;
    }
    return true;
}

__device__ inline bool fcr_eval(const double* F, double mu, double lam, double& psi, double* P) {
    double C[9], R[9];
    cof3(F, C);
    const double J = F[0] * C[0] + F[1] * C[1] + F[2] * C[2];
    if (!(J > 0.0) || !polar_rotation(F, R)) return false;
    double d2 = 0.0;
    for (int i = 0; i < 9; ++i) d2 += (F[i] - R[i]) * (F[i] - R[i]);
    psi = mu * d2 + 0.5 * lam * (J - 1.0) * (J - 1.0);
    if (P)
        for (int i = 0; i < 9; ++i) P[i] = 2.0 * mu * (F[i] - R[i]) + lam * (J - 1.0) * C[i];
    return true;
}

// F-space Hessian of the fixed-corotated density, column (a, b) for
// dF = e_a e_b^T:  2 mu (dF - dR) + lam cof(F) cof(F)_ab + lam (J - 1) dcof,
// with dcof_ij = eps_iak eps_jbn F_kn and the rotation's differential
// dR = R [w]x, w = (tr(S) I - S)^-1 axial(R^T dF - dF^T R), S = R^T F (from
// R^T dF - dF^T R = w S + S w for the skew w = R^T dR); symmetrised, then
// projected onto the PSD cone by Jacobi rotations.  J > 0 is assumed.
template <class T>
__device__ inline void fcr_hessian_projected(const double* F, double mu, double lam, SMat<9, T> H, T* W) {
    double C[9], R[9], S[9], M[9], Mi[9];
    cof3(F, C);
    const double J = F[0] * C[0] + F[1] * C[1] + F[2] * C[2];
    polar_rotation(F, R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
            for (int k = 0; k < 3; ++k) v += R[3 * k + i] * F[3 * k + j];
            S[3 * i + j] = v;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j) S[3 * i + j] = S[3 * j + i] = 0.5 * (S[3 * i + j] + S[3 * j + i]);
    const double trS = S[0] + S[4] + S[8];
    for (int i = 0; i < 9; ++i) M[i] = (i % 4 == 0 ? trS : 0.0) - S[i];
    double Cm[9];
    cof3(M, Cm);
    const double detM = M[0] * Cm[0] + M[1] * Cm[1] + M[2] * Cm[2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Mi[3 * i + j] = Cm[3 * j + i] / detM;  // inverse = adjugate / det
    double Hd[81];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            // K = A - A^T with A = R^T dF, A_pq = R_ap delta_qb
            double K[9];
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) K[3 * p + q] = (q == b ? R[3 * a + p] : 0.0) - (p == b ? R[3 * a + q] : 0.0);
            const double k[3] = {K[7], K[2], K[3]};  // axial vector of the skew K
            double w[3];
            for (int i = 0; i < 3; ++i) w[i] = Mi[3 * i] * k[0] + Mi[3 * i + 1] * k[1] + Mi[3 * i + 2] * k[2];
            const double Om[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double dR = 0.0;
                    for (int k2 = 0; k2 < 3; ++k2) dR += R[3 * i + k2] * Om[3 * k2 + j];
                    double dcof = 0.0;
                    for (int k2 = 0; k2 < 3; ++k2)
                        for (int n = 0; n < 3; ++n) dcof += lc(i, a, k2) * lc(j, b, n) * F[3 * k2 + n];
                    const double dF = (i == a && j == b) ? 1.0 : 0.0;
                    Hd[9 * (3 * i + j) + 3 * a + b] =
                        2.0 * mu * (dF - dR) + lam * C[3 * i + j] * C[3 * a + b] + lam * (J - 1.0) * dcof;
                }
        }
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) H(r, c) = (T)(0.5 * (Hd[9 * r + c] + Hd[9 * c + r]));
    psd_project<9, T>(H, SMat<9, T>{W, 1});
}

__device__ __forceinline__ void tet_F(const Geo& G, const double* x, int t, double* F, int4& T) {
    T = G.tets[t];
    V3 x0 = ld3(x + 3 * (size_t)T.x), x1 = ld3(x + 3 * (size_t)T.y), x2 = ld3(x + 3 * (size_t)T.z),
       x3 = ld3(x + 3 * (size_t)T.w);
    V3 e[3] = {x1 - x0, x2 - x0, x3 - x0};
    const double* Dm = G.Dminv + 9 * (size_t)t;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            F[3 * r + c] = comp(e[0], r) * Dm[c] + comp(e[1], r) * Dm[3 + c] + comp(e[2], r) * Dm[6 + c];
}

constexpr int EL_T = 64;

// Elastic gradient (FP64) and F-space-projected Hessian (in T) per tet: 16
// blocks (3x3) of h^2 V B^T P(H_F) B and 12 gradient entries h^2 V B^T vec(P)
// into staging.
template <class T>
__global__ void __launch_bounds__(EL_T) k_elastic_gh(Geo G, const double* x, T* stage_blk, double* stage_g) {
    extern __shared__ unsigned char smraw[];
    T* sm = (T*)smraw;
    int t = blockIdx.x * EL_T + threadIdx.x;
    if (t >= G.n_tets) return;
    if (G.env_done && G.env_done[G.node_env[G.tets[t].x]]) return;
    SMat<9, T> H{sm + threadIdx.x, EL_T};
    double F[9], P[9], psi;
    int4 Tt;
    tet_F(G, x, t, F, Tt);
    if (G.tmodel[t] == 1) {
        T W[81];
        stvk_eval(F, G.tmu[t], G.tlam[t], psi, P);
        stvk_hessian_projected<T>(F, G.tmu[t], G.tlam[t], H, W);
    } else if (G.tmodel[t] == 2) {
        if (!fcr_eval(F, G.tmu[t], G.tlam[t], psi, P)) {
            for (int i = 0; i < 16 * 9; ++i) stage_blk[(size_t)t * 144 + i] = T(0);
            for (int i = 0; i < 12; ++i) stage_g[(size_t)t * 12 + i] = 0.0;
            return;
        }
        T W[81];
        fcr_hessian_projected<T>(F, G.tmu[t], G.tlam[t], H, W);
    } else {
        if (!nh_eval(F, G.tmu[t], G.tlam[t], psi, P, nullptr)) {
            // inverted (never reached at an accepted iterate): zero contribution
            for (int i = 0; i < 16 * 9; ++i) stage_blk[(size_t)t * 144 + i] = T(0);
            for (int i = 0; i < 12; ++i) stage_g[(size_t)t * 12 + i] = 0.0;
            return;
        }
        nh_hessian_projected<T>(F, G.tmu[t], G.tlam[t], H);
    }
    double D[4][3];
    dF_coef(G.Dminv + 9 * (size_t)t, D);
    double w = G.h * G.h * G.tvol[t];
    for (int v = 0; v < 4; ++v)
        for (int r = 0; r < 3; ++r) {
            double s = 0.0;
            for (int c = 0; c < 3; ++c) s += P[3 * r + c] * D[v][c];
            stage_g[(size_t)t * 12 + 3 * v + r] = w * s;
        }
    T Dt[4][3];
    for (int v = 0; v < 4; ++v)
        for (int c = 0; c < 3; ++c) Dt[v][c] = (T)D[v][c];
    T wt = (T)w;
    for (int v = 0; v < 4; ++v)
        for (int u = 0; u < 4; ++u) {
            T* out = stage_blk + ((size_t)t * 16 + 4 * v + u) * 9;
            for (int r = 0; r < 3; ++r)
                for (int s = 0; s < 3; ++s) {
                    T acc = 0;
                    for (int c = 0; c < 3; ++c) {
                        T inner = 0;
                        for (int d = 0; d < 3; ++d) inner += H(3 * r + c, 3 * s + d) * Dt[u][d];
                        acc += Dt[v][c] * inner;
                    }
                    out[3 * r + s] = wt * acc;
                }
        }
}

// soft inertia (Eq. 1) and elasticity (Eq. 1, h^2 Phi) energies per env
__global__ void k_soft_energy(Geo G, const double* x, const double* xhat, double* part) {
    int env = blockIdx.y;
    if (env_is_done(G, env)) return;
    int n0 = G.env_node_start[env], n1 = G.env_node_start[env + 1];
    chunk_sum(
        n0, n1,
        [&](int n) -> double {
            double m = G.node_mass[n];
            if (m == 0.0) return 0.0;
            V3 d = ld3(x + 3 * (size_t)n) - ld3(xhat + 3 * (size_t)n);
            double e = 0.5 * m * dot(d, d);
            if (G.spring_k && G.spring_k[n] > 0.0) {
                // spring constraint: h^2 k |x - x_target|^2
                V3 r = ld3(x + 3 * (size_t)n) - ld3(G.spring_x + 3 * (size_t)n);
                e += G.h * G.h * G.spring_k[n] * dot(r, r);
            }
            return e;
        },
        part_slot(part, ET_INERTIA, G.n_envs, env));
    int t0 = G.env_tet_start[env], t1 = G.env_tet_start[env + 1];
    chunk_sum(
        t0, t1,
        [&](int t) -> double {
            double F[9], psi;
            int4 T;
            tet_F(G, x, t, F, T);
            if (G.tmodel[t] == 1)
                stvk_eval(F, G.tmu[t], G.tlam[t], psi, nullptr);
            else if (G.tmodel[t] == 2) {
                if (!fcr_eval(F, G.tmu[t], G.tlam[t], psi, nullptr)) return INFINITY;
            } else if (!nh_eval(F, G.tmu[t], G.tlam[t], psi, nullptr, nullptr))
                return INFINITY;
            return G.h * G.h * G.tvol[t] * psi;
        },
        part_slot(part, ET_ELASTIC, G.n_envs, env));
}

// gradient of soft nodes: inertia + gather of the incident tets' staging
__global__ void k_soft_grad(Geo G, const double* x, const double* xhat, const double* stage_g, double* g) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.n_nodes) return;
    double m = G.node_mass[n];
    if (m == 0.0) return;  // affine node
    if (env_is_done(G, G.node_env[n])) return;
    V3 d = ld3(x + 3 * (size_t)n) - ld3(xhat + 3 * (size_t)n);
    V3 s = m * d;
    if (G.spring_k && G.spring_k[n] > 0.0)
        s = s + (2.0 * G.h * G.h * G.spring_k[n]) * (ld3(x + 3 * (size_t)n) - ld3(G.spring_x + 3 * (size_t)n));
    for (int k = G.node_tet_ptr[n]; k < G.node_tet_ptr[n + 1]; ++k) {
        int e = G.node_tet_idx[k];  // tet * 4 + local
        s = s + ld3(stage_g + 3 * (size_t)e);
    }
    if (G.node_fixed[n]) s = v3(0, 0, 0);
    st3(g + 3 * (size_t)n, s);
}

// ---------------------------------------------------------------------------
// Affine bodies (Eq. 2, Eq. 13) in the centred column form.
// ---------------------------------------------------------------------------
struct AffKin {
    const double* qtarget;  // 12 per body, caller's row form
    const double* lamA;     // 12 per body
};

// energy of one affine body (inertia + orthogonality + kinematic AL)
__device__ inline double affine_energy(const Geo& G, const double* x, const double* xhat, AffKin K, int b) {
    int mode = G.aff_mode[b];
    if (mode == 1) return 0.0;
    int n0 = G.aff_node0[b];
    V3 c[4], ch[4];
    for (int j = 0; j < 4; ++j) {
        c[j] = ld3(x + 3 * (size_t)(n0 + j));
        ch[j] = ld3(xhat + 3 * (size_t)(n0 + j));
    }
    const double* S = G.aff_S + 9 * (size_t)b;
    double m = G.aff_m[b];
    V3 dp = c[0] - ch[0];
    double E = 0.5 * m * dot(dp, dp);
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) E += 0.5 * S[3 * j + k] * dot(c[1 + j] - ch[1 + j], c[1 + k] - ch[1 + k]);
    double o = 0.0;
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
            double gjk = dot(c[1 + j], c[1 + k]) - (j == k ? 1.0 : 0.0);
            o += gjk * gjk;
        }
    E += G.h * G.h * G.aff_stiff[b] * G.aff_vol[b] * o;
    if (mode == 2) {
        const double* qt = K.qtarget + 12 * (size_t)b;
        const double* la = K.lamA + 12 * (size_t)b;
        double kA = 1e3 * m, sm = sqrt(m);
        const double* com = G.aff_com + 3 * (size_t)b;
        // caller-frame translation p = p' - A com ; A rows a_i = (c1_i, c2_i, c3_i)
        V3 p = c[0] - (com[0] * c[1] + com[1] * c[2] + com[2] * c[3]);
        double q[12] = {p.x, p.y, p.z, c[1].x, c[2].x, c[3].x, c[1].y, c[2].y, c[3].y, c[1].z, c[2].z, c[3].z};
        for (int i = 0; i < 12; ++i) {
            double d = q[i] - qt[i];
            E += 0.5 * kA * d * d - sm * la[i] * d;
        }
    }
    return E;
}

__global__ void k_affine_energy(Geo G, const double* x, const double* xhat, AffKin K, double* part) {
    int env = blockIdx.y;
    if (env_is_done(G, env)) return;
    chunk_sum(
        G.env_aff_start[env], G.env_aff_start[env + 1],
        [&](int b) -> double { return affine_energy(G, x, xhat, K, b); }, part_slot(part, ET_AFFINE, G.n_envs, env));
}

constexpr int kAffBodies = 4;  // affine bodies per 64-thread block of k_affine_gh

// gradient (FP64, directly into g, the body's nodes only) and 16 Hessian
// blocks (in T), one affine body per half-warp: the 9x9 orthogonality
// Hessian (A-space) is built by lanes 0-8, one row each, and projected to PSD
// by the 16-lane parallel Jacobi (coop_psd9); lane 0 then assembles the
// blocks and the gradient.
template <class T>
__global__ void __launch_bounds__(kCoopLanes * kAffBodies) k_affine_gh(Geo G, const double* x, const double* xhat,
                                                                      AffKin K, T* stage_blk, double* g) {
    __shared__ T sP[kAffBodies][81];
    __shared__ T sV[kAffBodies][100];
    __shared__ T sL[kAffBodies][10];
    const int hw = threadIdx.x / kCoopLanes, lane = threadIdx.x & (kCoopLanes - 1);
    const unsigned mask = 0xFFFFu << (threadIdx.x & 16);
    const int b = blockIdx.x * kAffBodies + hw;
    if (b >= G.n_aff) return;  // the whole half-warp
    const int mode = G.aff_mode[b];
    const int n0 = G.aff_node0[b];
    if (env_is_done(G, G.node_env[n0])) return;
    T* blk = stage_blk + (size_t)b * 144;
    if (mode == 1) {
        for (int i = lane; i < 144; i += kCoopLanes) blk[i] = T(0);
        if (lane < 4) st3(g + 3 * (size_t)(n0 + lane), v3(0, 0, 0));
        return;
    }
    V3 c[4];
    for (int j = 0; j < 4; ++j) c[j] = ld3(x + 3 * (size_t)(n0 + j));
    // orthogonality: Phi = sum_jk (c_j . c_k - delta_jk)^2, its Hessian in
    // A = (c_1, c_2, c_3) built by rows (lane r < 9: row r = 3 i + a)
    const double w = G.h * G.h * G.aff_stiff[b] * G.aff_vol[b];
    double Gm[3][3];
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) Gm[j][k] = dot(c[1 + j], c[1 + k]) - (j == k ? 1.0 : 0.0);
    T a[kCoopN];
    for (int q = 0; q < kCoopN; ++q) a[q] = T(0);
    if (lane < 9) {
        const int i = lane / 3, al = lane - 3 * i;
        for (int l = 0; l < 3; ++l)
            for (int bb = 0; bb < 3; ++bb) {
                double v = comp(c[1 + l], al) * comp(c[1 + i], bb);
                if (al == bb) v += Gm[i][l];
                if (i == l)
                    v += comp(c[1], al) * comp(c[1], bb) + comp(c[2], al) * comp(c[2], bb) +
                         comp(c[3], al) * comp(c[3], bb);
                a[3 * l + bb] = (T)(4.0 * w * v);
            }
    }
    coop_psd9<T>(a, sP[hw], sV[hw], sL[hw], mask);
    if (lane != 0) return;
    const T* P = sP[hw];
    for (int i = 0; i < 144; ++i) blk[i] = T(0);
    V3 ch[4];
    for (int j = 0; j < 4; ++j) ch[j] = ld3(xhat + 3 * (size_t)(n0 + j));
    const double* S = G.aff_S + 9 * (size_t)b;
    double m = G.aff_m[b];
    V3 gr[4];
    gr[0] = m * (c[0] - ch[0]);
    for (int j = 0; j < 3; ++j) {
        V3 sj = v3(0, 0, 0);
        for (int k = 0; k < 3; ++k) sj = sj + S[3 * j + k] * (c[1 + k] - ch[1 + k]);
        gr[1 + j] = sj;
    }
    // inertia blocks: (0,0) m I ; (j,k) S_jk I
    auto blk_add_diag = [&](int j, int k, double v) {
        T* o = blk + (4 * j + k) * 9;
        o[0] += (T)v;
        o[4] += (T)v;
        o[8] += (T)v;
    };
    blk_add_diag(0, 0, m);
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) blk_add_diag(1 + j, 1 + k, S[3 * j + k]);
    for (int i = 0; i < 3; ++i) {
        V3 si = v3(0, 0, 0);
        for (int k = 0; k < 3; ++k) si = si + Gm[i][k] * c[1 + k];
        gr[1 + i] = gr[1 + i] + (4.0 * w) * si;
    }
    for (int i = 0; i < 3; ++i)
        for (int l = 0; l < 3; ++l) {
            T* o = blk + (4 * (1 + i) + (1 + l)) * 9;
            for (int al = 0; al < 3; ++al)
                for (int bb = 0; bb < 3; ++bb) o[3 * al + bb] += P[9 * (3 * i + al) + 3 * l + bb];
        }
    if (mode == 2) {
        const double* qt = K.qtarget + 12 * (size_t)b;
        const double* la = K.lamA + 12 * (size_t)b;
        double kA = 1e3 * m, sm_ = sqrt(m);
        const double* com = G.aff_com + 3 * (size_t)b;
        double wo[4] = {1.0, -com[0], -com[1], -com[2]};
        V3 p = c[0] - (com[0] * c[1] + com[1] * c[2] + com[2] * c[3]);
        V3 fp = kA * (p - ld3(qt)) - sm_ * ld3(la);
        for (int j = 0; j < 4; ++j) gr[j] = gr[j] + wo[j] * fp;
        for (int j = 0; j < 4; ++j)
            for (int l = 0; l < 4; ++l) blk_add_diag(j, l, kA * wo[j] * wo[l]);
        for (int k = 0; k < 3; ++k) {
            // column k of the target A (rows a_i at qt[3 + 3 i]) and of Lambda
            V3 ct = v3(qt[3 + k], qt[6 + k], qt[9 + k]);
            V3 lk = v3(la[3 + k], la[6 + k], la[9 + k]);
            gr[1 + k] = gr[1 + k] + (kA * (c[1 + k] - ct) - sm_ * lk);
            blk_add_diag(1 + k, 1 + k, kA);
        }
    }
    for (int j = 0; j < 4; ++j) st3(g + 3 * (size_t)(n0 + j), gr[j]);
}

// ---------------------------------------------------------------------------
// Contact barrier (Eq. 4-8) per active pair: gradient and projected Hessian
// in the 12-dim stencil space.
// ---------------------------------------------------------------------------

__device__ __forceinline__ double pair_eps_x(const Geo& G, const PairRec& r) {
    if (!r.is_ee) return 0.0;
    V3 a = ld3(G.sv_rest + 3 * (size_t)r.s[1]) - ld3(G.sv_rest + 3 * (size_t)r.s[0]);
    V3 b = ld3(G.sv_rest + 3 * (size_t)r.s[3]) - ld3(G.sv_rest + 3 * (size_t)r.s[2]);
    return 1e-3 * dot(a, a) * dot(b, b);
}

// Barrier gradient (FP64) and PSD-projected Hessian (T) of many pairs, in
// two launches so that each runs within its own register budget:
//   raw      one pair per thread: distance type, barrier value and FP64
//            gradient, and the unprojected 12x12 slot-space Hessian written
//            in place of the pair's output block; flag 1 marks a block to
//            project (0: inactive pair);
//   project  one pair per half-warp at 64 registers per thread (four times
//            the resident warps of the raw pass): the block into shared
//            memory, then the 16-lane Jacobi projection of barrier_coop.cuh
//            back into the output block.
// The arithmetic and its order are those of the one-pair-per-half-warp form
// below, so both give the same bits.  load(i, x, is_ee, eps_x, kappa)
// supplies pair i's stencil.  A Hessian outside T's range (degenerate
// stencil) is left out; the pair still contributes its exact FP64 gradient.
constexpr int kRawThreads = 32;  // one warp per block: 32 Hessian blocks in shared memory
constexpr int kRawPad = 145;     // per-pair stride in shared memory: odd, so the 32 lanes' slots fall in distinct banks
constexpr int kProjPairs = 8;    // pairs per 128-thread block of the projection

template <class T, class Load>
__device__ __forceinline__ void barrier_gh_raw(int n, const Load& load, double dhat, T* pH, double* pG, double* pE,
                                               int* flag) {
    __shared__ T sH[kRawThreads][kRawPad];
    const int lane = threadIdx.x;
    const int base = blockIdx.x * kRawThreads;
    const int i = base + lane;
    if (i < n) {
        V3 x[4];
        int is_ee;
        double eps_x, kap, E = 0.0, g12[12];
        load(i, x, is_ee, eps_x, kap);
        const int act =
            pair_barrier<T>(x, is_ee != 0, dhat, kap, eps_x, E, g12, SMat<12, T>{sH[lane], 1}, true);
        for (int a = 0; a < 12; ++a) pG[(size_t)i * 12 + a] = act ? g12[a] : 0.0;
        if (pE) pE[i] = act ? E : 0.0;
        flag[i] = act ? 1 : 0;
    }
    __syncwarp();
    // the warp's blocks are contiguous in pH: one coalesced sweep
    const int m = min(kRawThreads, n - base);
    for (int k = lane; k < 144 * m; k += kRawThreads) {
        const int p = k / 144;
        pH[(size_t)base * 144 + k] = sH[p][k - 144 * p];
    }
}

template <class T>
__device__ __forceinline__ void barrier_project_half(int n, double kap, const int* flag, T* pH) {
    __shared__ T sm[kProjPairs][kCoopSmem];
    const int grp = threadIdx.x / kCoopLanes, lane = threadIdx.x & (kCoopLanes - 1);
    const int i = blockIdx.x * kProjPairs + grp;
    if (i >= n) return;  // the whole half-warp
    const unsigned mask = 0xFFFFu << (threadIdx.x & 16);
    T* out = pH + (size_t)i * 144;
    T* H = sm[grp];
    const bool act = flag[i] == 1;
    bool finite = true;
    if (act)
        for (int e = lane; e < 144; e += kCoopLanes) {
            const T v = out[e];
            H[e] = v;
            finite &= isfinite(v);
        }
    finite = __all_sync(mask, finite);
    if (!act || !finite) {
        for (int e = lane; e < 144; e += kCoopLanes) out[e] = T(0);
        return;
    }
    __syncwarp(mask);
    coop_project<T>(H, H + 144, H + 244, kap, out, mask);
}

// Few pairs (an IPC step often has only hundreds): one pair per half-warp,
// lane 0 doing the FP64 part, so that many warps share the work.
template <class T>
__global__ void __launch_bounds__(kCoopLanes * kCoopPairs) k_barrier_gh_half(Geo G, const double* X,
                                                                            const PairRec* rec, int n,
                                                                            const double* kappa_env, T* pH,
                                                                            double* pG) {
    __shared__ T sm[kCoopPairs][kCoopSmem];
    const int grp = threadIdx.x / kCoopLanes, lane = threadIdx.x & (kCoopLanes - 1);
    const int i = blockIdx.x * kCoopPairs + grp;
    if (i >= n) return;  // the whole half-warp
    const unsigned mask = 0xFFFFu << (threadIdx.x & 16);
    T* H = sm[grp];
    int act = 0;
    double kap = 0.0;
    if (lane == 0) {
        PairRec r = rec[i];
        V3 x[4];
        for (int k = 0; k < 4; ++k) x[k] = ld3(X + 3 * (size_t)r.s[k]);
        kap = kappa_env[G.sv_env[r.s[0]]];
        double E, g12[12];
        act = pair_barrier<T>(x, r.is_ee != 0, G.dhat, kap, pair_eps_x(G, r), E, g12, SMat<12, T>{H, 1}, true);
        for (int a = 0; a < 12; ++a) pG[(size_t)i * 12 + a] = act ? g12[a] : 0.0;
        // a Hessian outside T's range (degenerate stencil) is left out: the
        // pair still contributes its exact FP64 gradient
        if (act) {
            bool finite = true;
            for (int a = 0; a < 144; ++a) finite &= isfinite(H[a]);
            if (!finite) act = 2;
        }
    }
    act = __shfl_sync(mask, act, 0, kCoopLanes);
    kap = __shfl_sync(mask, kap, 0, kCoopLanes);
    T* out = pH + (size_t)i * 144;
    if (act != 1) {
        for (int e = lane; e < 144; e += kCoopLanes) out[e] = T(0);
        return;
    }
    __syncwarp(mask);
    coop_project<T>(H, H + 144, H + 244, kap, out, mask);
}

// Many pairs: the two-launch form above.
constexpr int kSplitMinPairs = 16384;
template <class T>
__global__ void __launch_bounds__(kRawThreads) k_barrier_gh_raw(Geo G, const double* X, const PairRec* rec, int n,
                                                               const double* kappa_env, T* pH, double* pG,
                                                               int* flag) {
    auto load = [&](int i, V3* x, int& is_ee, double& eps_x, double& kap) {
        const PairRec r = rec[i];
        for (int k = 0; k < 4; ++k) x[k] = ld3(X + 3 * (size_t)r.s[k]);
        is_ee = r.is_ee;
        eps_x = pair_eps_x(G, r);
        kap = kappa_env[G.sv_env[r.s[0]]];
    };
    barrier_gh_raw<T>(n, load, G.dhat, pH, pG, nullptr, flag);
}

template <class T>
__global__ void __launch_bounds__(kCoopLanes * kProjPairs, 8) k_barrier_project(Geo G, const PairRec* rec, int n,
                                                                                 const double* kappa_env,
                                                                                 const int* flag, T* pH) {
    const int i = blockIdx.x * kProjPairs + (int)(threadIdx.x / kCoopLanes);
    const double kap = i < n ? kappa_env[G.sv_env[rec[i].s[0]]] : 0.0;
    barrier_project_half<T>(n, kap, flag, pH);
}

// barrier energy over a pair list per env (ranges from env_off)
__global__ void k_barrier_energy(Geo G, const double* X, const PairRec* rec, const uint32_t* env_off,
                                 const double* kappa_env, double* part) {
    int env = blockIdx.y;
    if (env_is_done(G, env)) return;
    double kap = kappa_env[env];
    chunk_sum(
        (int)env_off[env], (int)env_off[env + 1],
        [&](int i) -> double {
            PairRec r = rec[i];
            V3 x[4];
            for (int k = 0; k < 4; ++k) x[k] = ld3(X + 3 * (size_t)r.s[k]);
            return pair_barrier_energy(x, r.is_ee != 0, G.dhat, kap, pair_eps_x(G, r), nullptr);
        },
        part_slot(part, ET_BARRIER, G.n_envs, env));
}

// Contact force sensing: per body b (one block), the sum over b's surface
// vertices of the barrier gradient dB/dx_v of the active pairs of b's env,
// divided by h^2 (B is the h^2-scaled barrier of the incremental potential,
// so the result is in newtons; the force the contacts exert on the body is
// its negative).  Fixed-order block sum: bit-reproducible.
__global__ void k_body_contact_force(Geo G, const double* X, const PairRec* rec, const uint32_t* env_off,
                                     const int* body_env, const double* kappa_env, double inv_h2, double* force) {
    __shared__ double sh[32];
    const int b = blockIdx.x, e = body_env[b];
    const double kap = kappa_env[e];
    double f[3] = {0.0, 0.0, 0.0};
    for (int i = (int)env_off[e] + threadIdx.x; i < (int)env_off[e + 1]; i += blockDim.x) {
        const PairRec r = rec[i];
        bool touch = false;
        for (int k = 0; k < 4; ++k) touch |= G.sv_body[r.s[k]] == b;
        if (!touch) continue;
        V3 x[4];
        for (int k = 0; k < 4; ++k) x[k] = ld3(X + 3 * (size_t)r.s[k]);
        double E, g12[12];
        if (!pair_barrier<double>(x, r.is_ee != 0, G.dhat, kap, pair_eps_x(G, r), E, g12, SMat<12, double>{nullptr, 0},
                                  false))
            continue;
        for (int k = 0; k < 4; ++k)
            if (G.sv_body[r.s[k]] == b)
                for (int j = 0; j < 3; ++j) f[j] += g12[3 * k + j];
    }
    for (int j = 0; j < 3; ++j) {
        const double t = block_sum<128>(f[j], sh);
        if (threadIdx.x == 0) force[3 * b + j] = t * inv_h2;
    }
}

// ---------------------------------------------------------------------------
// Prismatic joint (paper Sec. "Joint Constraints"): constraint vector
//   c = ( vec(A1 B1 - A2 B2) , r x (A1 d1) ),  r = P1 + A1 u1 - P2 - A2 u2,
// zero when the relative orientation is the initial one and the joint point
// of body 2 stays on body 1's axis (with both initial A = I this is the
// paper's |A1 - A2|^2 + |((A1 c + p1) - (A2 c + p2)) x (A1 d)|^2 term).
// Energy kappa |c|^2 - lambda . c (augmented Lagrangian).  Jm: dc/dq over
// the 24 DOF, body 1's nodes (P, columns of A) then body 2's.
// ---------------------------------------------------------------------------
__device__ inline void joint_eval(const JointDev& J, const double* x, double* c, double (*Jm)[24]) {
    double P1[3], P2[3], A1[9], A2[9];
    for (int i = 0; i < 3; ++i) {
        P1[i] = x[3 * (size_t)J.n1 + i];
        P2[i] = x[3 * (size_t)J.n2 + i];
        for (int k = 0; k < 3; ++k) {
            A1[3 * i + k] = x[3 * (size_t)(J.n1 + 1 + k) + i];
            A2[3 * i + k] = x[3 * (size_t)(J.n2 + 1 + k) + i];
        }
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
            for (int k = 0; k < 3; ++k) v += A1[3 * i + k] * J.B1[3 * k + j] - A2[3 * i + k] * J.B2[3 * k + j];
            c[3 * i + j] = v;
        }
    double r[3], a[3];
    for (int i = 0; i < 3; ++i) {
        r[i] = P1[i] - P2[i];
        a[i] = 0.0;
        for (int k = 0; k < 3; ++k) {
            r[i] += A1[3 * i + k] * J.u1[k] - A2[3 * i + k] * J.u2[k];
            a[i] += A1[3 * i + k] * J.d1[k];
        }
    }
    c[9] = r[1] * a[2] - r[2] * a[1];
    c[10] = r[2] * a[0] - r[0] * a[2];
    c[11] = r[0] * a[1] - r[1] * a[0];
    if (!Jm) return;
    for (int m = 0; m < 12; ++m)
        for (int q = 0; q < 24; ++q) Jm[m][q] = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                Jm[3 * i + j][3 + 3 * k + i] += J.B1[3 * k + j];
                Jm[3 * i + j][15 + 3 * k + i] -= J.B2[3 * k + j];
            }
    // d(r x a) = -[a]x dr + [r]x da
    const double Ax[9] = {0.0, -a[2], a[1], a[2], 0.0, -a[0], -a[1], a[0], 0.0};
    const double Rx[9] = {0.0, -r[2], r[1], r[2], 0.0, -r[0], -r[1], r[0], 0.0};
    for (int m = 0; m < 3; ++m)
        for (int i = 0; i < 3; ++i) {
            Jm[9 + m][i] = -Ax[3 * m + i];
            Jm[9 + m][12 + i] = Ax[3 * m + i];
            for (int k = 0; k < 3; ++k) {
                Jm[9 + m][3 + 3 * k + i] = -Ax[3 * m + i] * J.u1[k] + Rx[3 * m + i] * J.d1[k];
                Jm[9 + m][15 + 3 * k + i] = Ax[3 * m + i] * J.u2[k];
            }
        }
}

__device__ inline double joint_energy(const Geo& G, const double* x, int j) {
    const JointDev J = G.joints[j];
    double c[12];
    joint_eval(J, x, c, nullptr);
    double e = 0.0;
    for (int m = 0; m < 12; ++m) e += J.kappa * c[m] * c[m] - G.lamJ[12 * (size_t)j + m] * c[m];
    return e;
}

__global__ void k_joint_energy(Geo G, const double* x, double* part) {
    const int env = blockIdx.y;
    if (env_is_done(G, env)) return;
    chunk_sum(
        G.env_joint_start[env], G.env_joint_start[env + 1], [&](int j) -> double { return joint_energy(G, x, j); },
        part_slot(part, ET_JOINT, G.n_envs, env));
}

// gradient J^T (2 kappa c - lambda) added to the bodies' free nodes, and the
// Gauss-Newton Hessian 2 kappa J^T J (PSD by construction) as 8 x 8 node
// blocks into staging; one thread, joints in order (deterministic sums)
template <class T>
__global__ void k_joint_gh(Geo G, const double* x, T* stage, double* g) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int j = 0; j < G.n_joints; ++j) {
        const JointDev J = G.joints[j];
        if (env_is_done(G, G.node_env[J.n1])) continue;
        double c[12], Jm[12][24], w[12];
        joint_eval(J, x, c, Jm);
        for (int m = 0; m < 12; ++m) w[m] = 2.0 * J.kappa * c[m] - G.lamJ[12 * (size_t)j + m];
        for (int q = 0; q < 24; ++q) {
            const bool body2 = q >= 12;
            if (body2 ? J.fix2 : J.fix1) continue;
            double v = 0.0;
            for (int m = 0; m < 12; ++m) v += Jm[m][q] * w[m];
            const int n = (body2 ? J.n2 : J.n1) + (q % 12) / 3;
            g[3 * (size_t)n + q % 3] += v;
        }
        T* out = stage + (size_t)j * 64 * 9;
        for (int a = 0; a < 8; ++a)
            for (int b = 0; b < 8; ++b)
                for (int r = 0; r < 3; ++r)
                    for (int cc = 0; cc < 3; ++cc) {
                        double v = 0.0;
                        for (int m = 0; m < 12; ++m) v += Jm[m][3 * a + r] * Jm[m][3 * b + cc];
                        out[(8 * a + b) * 9 + 3 * r + cc] = (T)(2.0 * J.kappa * v);
                    }
    }
}

// AL round test: |c| of the rotation part above tol_rel h, or of the slide
// part above the env's step tolerance, asks for another round
__global__ void k_joint_check(Geo G, const double* x, const double* tol_env, double tol_rel, int* need_env) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= G.n_joints) return;
    const JointDev J = G.joints[j];
    double c[12];
    joint_eval(J, x, c, nullptr);
    double mr = 0.0, ms = 0.0;
    for (int m = 0; m < 9; ++m) mr = fmax(mr, fabs(c[m]));
    for (int m = 9; m < 12; ++m) ms = fmax(ms, fabs(c[m]));
    if (mr > tol_rel * G.h || ms > tol_env[J.env]) atomicMax(&need_env[J.env], 1);
}

// multiplier update lambda <- lambda - 2 kappa c for envs that need a round
__global__ void k_joint_update(Geo G, const double* x, double* lamJ, const int* need_env) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= G.n_joints) return;
    const JointDev J = G.joints[j];
    if (!need_env[J.env]) return;
    double c[12];
    joint_eval(J, x, c, nullptr);
    for (int m = 0; m < 12; ++m) lamJ[12 * (size_t)j + m] -= 2.0 * J.kappa * c[m];
}

// ---------------------------------------------------------------------------
// Lagged friction (Eq. 9-10)
// ---------------------------------------------------------------------------
struct Lag {
    const PairRec* rec;
    const double* w;   // 4 per pair: Delta = sum w_k (x_k - x_k^t)
    const double* n;   // 3 per pair: unit normal at x^t
    const double* c;   // mu * lambda
    const uint32_t* env_off;
    int n_pairs;
};

// closest-point weights, normal and normal-force magnitude at x^t
__global__ void k_lag_friction(Geo G, const double* X, const PairRec* rec, int n, const double* kappa_env,
                               double* w_out, double* n_out, double* c_out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PairRec r = rec[i];
    V3 x[4];
    for (int k = 0; k < 4; ++k) x[k] = ld3(X + 3 * (size_t)r.s[k]);
    DistInfo di = classify(x, r.is_ee != 0);
    double d = sqrt(di.d2);
    V3 dv = v3(0, 0, 0);
    for (int k = 0; k < 4; ++k) dv = dv + di.w[k] * x[k];
    double dl = sqrt(dot(dv, dv));
    V3 nn = (1.0 / dl) * dv;
    double e = 1.0;
    double eps = pair_eps_x(G, r);
    if (r.is_ee && eps > 0.0) {
        V3 cr = cross(x[1] - x[0], x[3] - x[2]);
        double c = dot(cr, cr);
        if (c < eps) e = (c / eps) * (2.0 - c / eps);
    }
    double b, b1, b2;
    barrier_d012(d, G.dhat, b, b1, b2);
    int env = G.sv_env[r.s[0]];
    double lam = kappa_env[env] * e * fabs(b1);
    int ba = G.sv_body[r.s[0]], bb = G.sv_body[r.s[r.is_ee ? 2 : 1]];
    double mu = fmin(G.body_mu[ba], G.body_mu[bb]);
    for (int k = 0; k < 4; ++k) w_out[(size_t)i * 4 + k] = di.w[k];
    st3(n_out + 3 * (size_t)i, nn);
    c_out[i] = mu * lam;
}

__device__ __forceinline__ double f0_mollifier(double y, double eh) {
    if (y >= eh) return y;
    return -y * y * y / (3.0 * eh * eh) + y * y / eh + eh / 3.0;
}

// tangential displacement u = (I - n n^T) Delta of a lagged pair
__device__ __forceinline__ V3 lag_u(const double* X, const double* Xt, const Lag& L, int i) {
    PairRec r = L.rec[i];
    V3 D = v3(0, 0, 0);
    for (int k = 0; k < 4; ++k) {
        double w = L.w[(size_t)i * 4 + k];
        D = D + w * (ld3(X + 3 * (size_t)r.s[k]) - ld3(Xt + 3 * (size_t)r.s[k]));
    }
    V3 n = ld3(L.n + 3 * (size_t)i);
    return D - dot(n, D) * n;
}

__global__ void k_friction_energy(Geo G, const double* X, const double* Xt, Lag L, double* part) {
    int env = blockIdx.y;
    if (env_is_done(G, env)) return;
    double eh = G.eps_v * G.h;
    chunk_sum(
        (int)L.env_off[env], (int)L.env_off[env + 1],
        [&](int i) -> double {
            V3 u = lag_u(X, Xt, L, i);
            return L.c[i] * f0_mollifier(sqrt(dot(u, u)), eh);
        },
        part_slot(part, ET_FRICTION, G.n_envs, env));
}

// friction gradient and Hessian (PSD by construction) in stencil space
template <class T>
__global__ void k_friction_gh(Geo G, const double* X, const double* Xt, Lag L, T* pH, double* pG) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n_pairs) return;
    if (env_is_done(G, G.sv_env[L.rec[i].s[0]])) return;  // k_contact_count drops the record
    double eh = G.eps_v * G.h;
    V3 u = lag_u(X, Xt, L, i);
    V3 n = ld3(L.n + 3 * (size_t)i);
    double y = sqrt(dot(u, u));
    double c = L.c[i];
    double a1, a2, f1y;
    if (y >= eh) {
        a1 = 1.0 / y;
        a2 = -1.0 / (y * y * y);
        f1y = 1.0 / y;
    } else {
        a1 = 2.0 / eh - y / (eh * eh);
        a2 = y > 0.0 ? -1.0 / (eh * eh * y) : 0.0;
        f1y = a1;
    }
    double nv[3] = {n.x, n.y, n.z}, uv[3] = {u.x, u.y, u.z};
    double HD[9], gD[3];
    for (int a = 0; a < 3; ++a) {
        gD[a] = c * f1y * uv[a];
        for (int b = 0; b < 3; ++b)
            HD[3 * a + b] = c * (a1 * ((a == b ? 1.0 : 0.0) - nv[a] * nv[b]) + a2 * uv[a] * uv[b]);
    }
    const double* w = L.w + (size_t)i * 4;
    T* Ho = pH + (size_t)i * 144;
    double* Go = pG + (size_t)i * 12;
    for (int k = 0; k < 4; ++k)
        for (int a = 0; a < 3; ++a) {
            Go[3 * k + a] = w[k] * gD[a];
            for (int l = 0; l < 4; ++l)
                for (int b = 0; b < 3; ++b) Ho[12 * (3 * k + a) + 3 * l + b] = (T)(w[k] * w[l] * HD[3 * a + b]);
        }
}

}  // namespace zema
