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
    // count = false: a region around launches counted on their own (timed
    // as one when it is the selected kernel)
    explicit LaunchScope(const char* name, bool count = true);
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
// threads keeps one small matrix each without register spills.  T is double
// (FP64 path) or float (Hessians of the mixed-precision path).
// ---------------------------------------------------------------------------
template <int N, class T = double>
struct SMat {
    T* b;
    int ld;
    __device__ __forceinline__ T& operator()(int i, int j) const { return b[(i * N + j) * ld]; }
};

// convergence thresholds of the eigen-solver per precision
template <class T>
struct Eps;
template <>
struct Eps<double> {
    static constexpr double off2 = 1e-28;  // off-diagonal mass / diagonal mass at convergence
    static constexpr double skip = 1e-18;  // rotations below this relative size are skipped
};
template <>
struct Eps<float> {
    static constexpr float off2 = 1e-12f;
    static constexpr float skip = 1e-9f;
};

// Cholesky test: true iff A is positive definite (A untouched, W scratch).
template <int N, class T>
__device__ bool is_pd(SMat<N, T> A, SMat<N, T> W) {
    for (int i = 0; i < N; ++i)
        for (int j = 0; j <= i; ++j) W(i, j) = A(i, j);
    for (int j = 0; j < N; ++j) {
        T d = W(j, j);
        for (int k = 0; k < j; ++k) d -= W(j, k) * W(j, k);
        if (!(d > T(0))) return false;
        T l = sqrt(d);
        W(j, j) = l;
        T il = T(1) / l;
        for (int i = j + 1; i < N; ++i) {
            T s = W(i, j);
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
template <int N, class T>
__device__ void psd_project(SMat<N, T> A, SMat<N, T> V) {
    if (is_pd<N, T>(A, V)) return;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) V(i, j) = (i == j) ? T(1) : T(0);
    for (int sweep = 0; sweep < 30; ++sweep) {
        T off = 0, diag = 0;
        for (int i = 0; i < N; ++i) {
            diag += A(i, i) * A(i, i);
            for (int j = i + 1; j < N; ++j) off += A(i, j) * A(i, j);
        }
        // off-diagonal mass at the rounding floor of T: converged (cyclic
        // Jacobi converges quadratically; a tighter test would never be met)
        if (off <= Eps<T>::off2 * diag) break;
        bool rotated = false;
        for (int p = 0; p < N - 1; ++p)
            for (int q = p + 1; q < N; ++q) {
                T apq = A(p, q);
                T app = A(p, p), aqq = A(q, q);
                if (fabs(apq) <= Eps<T>::skip * sqrt(fabs(app * aqq)) || apq == T(0)) continue;
                rotated = true;
                // rotation angle that zeroes A(p, q)
                T tau = (aqq - app) / (T(2) * apq);
                T t = copysign(T(1), tau) / (fabs(tau) + sqrt(T(1) + tau * tau));
                T c = rsqrt(T(1) + t * t);
                T s = t * c;
                for (int k = 0; k < N; ++k) {
                    T akp = A(k, p), akq = A(k, q);
                    A(k, p) = c * akp - s * akq;
                    A(k, q) = s * akp + c * akq;
                }
                for (int k = 0; k < N; ++k) {
                    T apk = A(p, k), aqk = A(q, k);
                    A(p, k) = c * apk - s * aqk;
                    A(q, k) = s * apk + c * aqk;
                }
                for (int k = 0; k < N; ++k) {
                    T vkp = V(k, p), vkq = V(k, q);
                    V(k, p) = c * vkp - s * vkq;
                    V(k, q) = s * vkp + c * vkq;
                }
            }
        if (!rotated) break;
    }
    // A <- V max(L, 0) V^T ; eigenvalues are on A's diagonal
    T lam[N];
#pragma unroll
    for (int i = 0; i < N; ++i) lam[i] = fmax(A(i, i), T(0));
    for (int i = 0; i < N; ++i)
        for (int j = i; j < N; ++j) {
            T s = 0;
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
