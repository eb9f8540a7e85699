// Shared device helpers of the zema CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <string>

namespace zema {

// ---------------------------------------------------------------------------
// Error plumbing: internal code throws ZemaError; the C ABI catches it.
// ---------------------------------------------------------------------------
struct ZemaError {
    int status;
    std::string msg;
};

#define ZCHECK(call)                                                                                 \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            throw ::zema::ZemaError{3 /*ZEMA_ERR_CUDA*/,                                             \
                                    std::string(#call) + ": " + cudaGetErrorString(e_)};             \
    } while (0)

#define ZLAUNCH() ZCHECK(cudaGetLastError())

// Every kernel launch of the library goes through ZL, which counts it
// (zema_launch_count reports the total) and, when that kernel is the one
// selected by zema_profile_kernel, brackets it with CUDA events on the
// current stream.  A launch site may declare the launch's algorithmic bytes
// beforehand with alg_bytes_hint().
long long& launch_counter();
struct LaunchScope {
    bool timed;
    explicit LaunchScope(const char* name);
    ~LaunchScope();
};
void set_current_stream(cudaStream_t st);
void alg_bytes_hint(double bytes);
// adds algorithmic bytes to the selected kernel after the fact (iterative kernels)
void alg_bytes_add(const char* name, double bytes);
#define ZL(kernel, ...) ::zema::LaunchScope(#kernel), kernel<<<__VA_ARGS__>>>

constexpr int kChunks = 32;   // blocks per environment in segmented reductions
constexpr int kRedThreads = 256;

__host__ __device__ inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// 3-vector helpers on plain double arrays
// ---------------------------------------------------------------------------
struct V3 {
    double x, y, z;
};
__device__ __forceinline__ V3 v3(double a, double b, double c) { return V3{a, b, c}; }
__device__ __forceinline__ V3 ld3(const double* p) { return V3{p[0], p[1], p[2]}; }
__device__ __forceinline__ void st3(double* p, V3 a) {
    p[0] = a.x;
    p[1] = a.y;
    p[2] = a.z;
}
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(double s, V3 a) { return V3{s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double comp(V3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

// ---------------------------------------------------------------------------
// Symmetric N x N matrices held per thread in shared memory with a stride:
// element (i, j) lives at base[(i * N + j) * ld].  Used so that a block of
// threads keeps one small matrix each without register spills.
// ---------------------------------------------------------------------------
template <int N>
struct SMat {
    double* b;
    int ld;
    __device__ __forceinline__ double& operator()(int i, int j) const { return b[(i * N + j) * ld]; }
};

// Cholesky test: true iff A is positive definite (A untouched, W scratch).
template <int N>
__device__ bool is_pd(SMat<N> A, SMat<N> W) {
    for (int i = 0; i < N; ++i)
        for (int j = 0; j <= i; ++j) W(i, j) = A(i, j);
    for (int j = 0; j < N; ++j) {
        double d = W(j, j);
        for (int k = 0; k < j; ++k) d -= W(j, k) * W(j, k);
        if (!(d > 0.0)) return false;
        double l = sqrt(d);
        W(j, j) = l;
        double il = 1.0 / l;
        for (int i = j + 1; i < N; ++i) {
            double s = W(i, j);
            for (int k = 0; k < j; ++k) s -= W(i, k) * W(j, k);
            W(i, j) = s * il;
        }
    }
    return true;
}

// Projects the symmetric A onto the PSD cone in place: eigen-decomposition
// by cyclic Jacobi rotations, negative eigenvalues clamped to zero.
// V is scratch of the same shape.  A matrix that is already positive
// definite (checked by Cholesky) is left unchanged.
template <int N>
__device__ void psd_project(SMat<N> A, SMat<N> V) {
    if (is_pd<N>(A, V)) return;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) V(i, j) = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < N; ++i) {
            diag += A(i, i) * A(i, i);
            for (int j = i + 1; j < N; ++j) off += A(i, j) * A(i, j);
        }
        // off-diagonal mass below (1e-14)^2 of the diagonal: converged to
        // round-off (cyclic Jacobi converges quadratically; a tighter test
        // would never be met in FP64)
        if (off <= 1e-28 * diag) break;
        bool rotated = false;
        for (int p = 0; p < N - 1; ++p)
            for (int q = p + 1; q < N; ++q) {
                double apq = A(p, q);
                double app = A(p, p), aqq = A(q, q);
                if (fabs(apq) <= 1e-18 * sqrt(fabs(app * aqq)) || apq == 0.0) continue;
                rotated = true;
                // rotation angle that zeroes A(p, q)
                double tau = (aqq - app) / (2.0 * apq);
                double t = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = rsqrt(1.0 + t * t);
                double s = t * c;
                for (int k = 0; k < N; ++k) {
                    double akp = A(k, p), akq = A(k, q);
                    A(k, p) = c * akp - s * akq;
                    A(k, q) = s * akp + c * akq;
                }
                for (int k = 0; k < N; ++k) {
                    double apk = A(p, k), aqk = A(q, k);
                    A(p, k) = c * apk - s * aqk;
                    A(q, k) = s * apk + c * aqk;
                }
                for (int k = 0; k < N; ++k) {
                    double vkp = V(k, p), vkq = V(k, q);
                    V(k, p) = c * vkp - s * vkq;
                    V(k, q) = s * vkp + c * vkq;
                }
            }
        if (!rotated) break;
    }
    // A <- V max(L, 0) V^T ; eigenvalues are on A's diagonal
    double lam[N];
#pragma unroll
    for (int i = 0; i < N; ++i) lam[i] = fmax(A(i, i), 0.0);
    for (int i = 0; i < N; ++i)
        for (int j = i; j < N; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += V(i, k) * lam[k] * V(j, k);
            A(i, j) = s;
            A(j, i) = s;
        }
}

// ---------------------------------------------------------------------------
// Block-wide sum with a fixed reduction tree (deterministic).
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (l < NT / 32) ? sh[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;  // valid in thread 0
}

__device__ __forceinline__ double block_max(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    }
    __syncthreads();
    return r;
}

// atomic min of a non-negative double through its bit pattern (order of
// non-negative IEEE doubles equals the order of their bits)
__device__ __forceinline__ void atomic_min_pos(double* addr, double v) {
    atomicMin(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------
// IPC barrier b(d) of Eq. 5 and its first two derivatives in d.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void barrier_d012(double d, double dh, double& b, double& b1, double& b2) {
    double u = d - dh;
    double L = log(d / dh);
    b = -u * u * L;
    b1 = -2.0 * u * L - u * u / d;
    b2 = -2.0 * L - 4.0 * u / d + u * u / (d * d);
}

}  // namespace zema
