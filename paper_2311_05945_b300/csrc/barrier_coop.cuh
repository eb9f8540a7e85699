// Barrier gradient and PSD-projected Hessian with 16 lanes per contact pair.
//
// A pair's projected Hessian is a long serial computation when one thread
// does it (hundreds of Jacobi rotations over a 9x9 matrix in shared memory),
// and an IPC step has only hundreds to a few thousand active pairs: one thread
// per pair leaves each SM with a handful of threads and the kernel runs at the
// latency of a single thread's chain.  Here a half-warp works on one pair:
//
//   lane 0    distance type, barrier value and FP64 gradient, and the 12x12
//             slot-space Hessian (arithmetic type T) into shared memory;
//   lanes 0-8 one row each of K = T H T^T (the 9x9 translation-free form:
//             every barrier term depends on the four points only through their
//             differences, see project_translation_free);
//   all       parallel cyclic Jacobi on K, rows in registers (lane i holds row
//             i of K and of the eigenvector matrix V), the 9 indices (padded
//             to 10) visited in round-robin order so that each round applies
//             5 disjoint rotations at once (9 rounds per sweep);
//   all       P = V max(L, 0) V^T and out = T^T P T, a few entries per lane.
#pragma once
#include "distance.cuh"

namespace zema {

constexpr int kCoopLanes = 16;
constexpr int kCoopPairs = 4;   // pairs per 64-thread block
constexpr int kCoopN = 10;      // 9 rows padded to an even count for the round-robin schedule
constexpr int kCoopSmem = 256;  // T values of shared memory per pair

template <class T>
struct CoopSweeps;
template <>
struct CoopSweeps<float> {
    static constexpr int n = 15;
};
template <>
struct CoopSweeps<double> {
    static constexpr int n = 30;
};

// a[i] for a runtime index i (selects; no local memory)
template <class T>
__device__ __forceinline__ T sel_row(const T (&a)[kCoopN], int i) {
    T r = a[0];
#pragma unroll
    for (int k = 1; k < kCoopN; ++k) r = (i == k) ? a[k] : r;
    return r;
}

template <class T>
__device__ __forceinline__ T hshfl(unsigned mask, T v, int src) {
    return __shfl_sync(mask, v, src, kCoopLanes);
}

// Round-robin schedule of 10 indices: in round r index 9 meets r and index
// (r + m) mod 9 meets (r - m) mod 9, m = 1..4.
__device__ __forceinline__ int rr_partner(int i, int r) {
    if (i == 9) return r;
    if (i == r) return 9;
    return (2 * r - i + 18) % 9;
}

// PSD part P = V max(L, 0) V^T of a symmetric 9x9 matrix A by the 16 lanes
// of a half-warp: lane i < 9 holds row i of A in a[0..8] (a[9] = 0, lanes
// 9-15 all zeros).  Parallel cyclic Jacobi with rows in registers; P goes to
// shared memory (81 values, row-major).  Vs (100 values) and lam (10) are
// shared scratch.
template <class T>
__device__ void coop_psd9(T (&a)[kCoopN], T* P, T* Vs, T* lam, unsigned mask) {
    const int lane = threadIdx.x & (kCoopLanes - 1);
    T v[kCoopN];
#pragma unroll
    for (int c = 0; c < kCoopN; ++c) v[c] = (c == lane) ? T(1) : T(0);
    for (int sweep = 0; sweep < CoopSweeps<T>::n; ++sweep) {
        // stop when the off-diagonal mass is at the rounding floor of T
        T dg = sel_row(a, lane), rowsq = 0;
#pragma unroll
        for (int c = 0; c < kCoopN; ++c) rowsq += a[c] * a[c];
        T off = lane < kCoopN ? rowsq - dg * dg : T(0), dia = lane < kCoopN ? dg * dg : T(0);
#pragma unroll
        for (int o = kCoopLanes / 2; o > 0; o >>= 1) {
            off += __shfl_xor_sync(mask, off, o, kCoopLanes);
            dia += __shfl_xor_sync(mask, dia, o, kCoopLanes);
        }
        if (off <= Eps<T>::off2 * dia) break;  // same decision in all 16 lanes
#pragma unroll
        for (int r = 0; r < 9; ++r) {
            const int j = lane < kCoopN ? rr_partner(lane, r) : lane;
            const int p = min(lane, j), q = max(lane, j);
            const T dl = sel_row(a, lane), aj = sel_row(a, j);
            const T app = hshfl(mask, dl, p & 15), aqq = hshfl(mask, dl, q & 15);
            const T apq = hshfl(mask, aj, p & 15);  // lane p's a(p, q): both lanes use the same value
            T c = T(1), s = T(0);
            if (lane < kCoopN && j != lane && apq != T(0) && !(fabs(apq) <= Eps<T>::skip * sqrt(fabs(app * aqq)))) {
                T tau = (aqq - app) / (T(2) * apq);
                T t = copysign(T(1), tau) / (fabs(tau) + sqrt(T(1) + tau * tau));
                c = T(1) / sqrt(T(1) + t * t);
                s = t * c;
            }
            // rows p and q of J^T A: exchange rows with the partner
            T pr[kCoopN];
#pragma unroll
            for (int cc = 0; cc < kCoopN; ++cc) pr[cc] = hshfl(mask, a[cc], j & 15);
            if (lane < kCoopN && j != lane) {
                const bool is_p = lane == p;
#pragma unroll
                for (int cc = 0; cc < kCoopN; ++cc) a[cc] = is_p ? c * a[cc] - s * pr[cc] : s * pr[cc] + c * a[cc];
            }
            // columns of (J^T A) J and V J: the round's 4 rotations off the padding index
#pragma unroll
            for (int m = 1; m <= 4; ++m) {
                const int i1 = (r + m) % 9, i2 = (r - m + 9) % 9;
                const int P1 = i1 < i2 ? i1 : i2, Q = i1 < i2 ? i2 : i1;
                const T cm = hshfl(mask, c, P1), sm = hshfl(mask, s, P1);
                T t1 = a[P1], t2 = a[Q];
                a[P1] = cm * t1 - sm * t2;
                a[Q] = sm * t1 + cm * t2;
                t1 = v[P1];
                t2 = v[Q];
                v[P1] = cm * t1 - sm * t2;
                v[Q] = sm * t1 + cm * t2;
            }
        }
    }
    // P = V max(L, 0) V^T
    if (lane < 9) {
        T l = sel_row(a, lane);
        lam[lane] = l > T(0) ? l : T(0);
#pragma unroll
        for (int c = 0; c < 9; ++c) Vs[10 * lane + c] = v[c];
    }
    __syncwarp(mask);
    for (int e = lane; e < 81; e += kCoopLanes) {
        const int i = e / 9, jj = e - 9 * i;
        T s = 0;
#pragma unroll
        for (int k = 0; k < 9; ++k) s += Vs[10 * i + k] * lam[k] * Vs[10 * jj + k];
        P[e] = s;
    }
    __syncwarp(mask);
}

// out = T^T P(scale T H T^T) T for the 12x12 slot-space Hessian H (row-major
// in shared memory; its storage is reused), by the 16 lanes of a half-warp.
// Vs (100 values) and lam (10) are shared scratch of the pair.
template <class T>
__device__ void coop_project(T* H, T* Vs, T* lam, double scale, T* out, unsigned mask) {
    const int lane = threadIdx.x & (kCoopLanes - 1);
    T a[kCoopN];
#pragma unroll
    for (int c = 0; c < kCoopN; ++c) a[c] = T(0);
    if (lane < 9) {
        // row lane = 3k + al of K: K(3k+al, 3l+b) = scale sum_ij T[k][i] T[l][j] H(3i+al, 3j+b)
        const int k = lane / 3, al = lane - 3 * k;
        T w[4][9];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int l = 0; l < 3; ++l)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    T s = 0;
#pragma unroll
                    for (int j = 0; j < 4; ++j) s += (T)tcoef(l, j) * H[(3 * i + al) * 12 + 3 * j + b];
                    w[i][3 * l + b] = s;
                }
        const T sc = (T)scale;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            T s = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) s += (T)tcoef(k, i) * w[i][c];
            a[c] = sc * s;
        }
    }
    __syncwarp(mask);  // every lane has read H: its storage now takes P
    coop_psd9<T>(a, H, Vs, lam, mask);
    for (int e = lane; e < 144; e += kCoopLanes) {
        const int row = e / 12, col = e - 12 * row;
        const int i = row / 3, al = row - 3 * i, jj = col / 3, b = col - 3 * jj;
        T s = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T t = 0;
#pragma unroll
            for (int l = 0; l < 3; ++l) t += (T)tcoef(l, jj) * H[(3 * k + al) * 9 + 3 * l + b];
            s += (T)tcoef(k, i) * t;
        }
        out[e] = s;
    }
}

}  // namespace zema
