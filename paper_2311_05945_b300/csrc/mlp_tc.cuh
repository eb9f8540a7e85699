// Fifth-generation tensor-core (tcgen05) product for the MLP's forward
// layers: Y (M x N) = X (M x K) W (K x N), BF16 operands, FP32 accumulation
// in tensor memory.
//
// A CTA (4 warps) computes 128-row tiles with all N <= 256 columns:
//   * X's 128 x K tile and W^T (N x K) sit in shared memory in the canonical
//     K-major layout without swizzle: 8-row x 16-byte core matrices, the
//     K-adjacent ones 128 B apart (leading byte offset), the row-group-
//     adjacent ones K/8 * 128 B apart (stride byte offset), written with
//     16-byte stores;
//   * warp 0 allocates N (rounded to a power of two, >= 32) TMEM columns;
//   * per tile one thread issues K/16 tcgen05.mma (M = 128, K = 16 each) and
//     commits them to an mbarrier; every thread waits on it with a bounded
//     spin (on timeout the kernel records an error flag and writes nothing);
//   * each warp reads its 32 accumulator rows (TMEM lanes 32w..32w+31) with
//     tcgen05.ld and applies the epilogue (bias, ReLU) of k_gemm_bf16;
//   * warp 0 frees the TMEM columns at the end.
#pragma once
#include "mlp.cuh"

namespace zema {

constexpr int kTcM = 128;
constexpr int kTcThreads = 128;
constexpr int kTcSpinLimit = 1 << 22;  // mbarrier polls (32 ns apart after the first 1024) before giving up

__device__ __forceinline__ uint32_t tc_smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared memory matrix descriptor: start address, leading / stride byte
// offsets (all in 16-byte units), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N / 8 and M / 16
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// byte offset of element (row, k) in a canonical K-major operand with kp
// (multiple of 16) columns
__device__ __forceinline__ uint32_t tc_off(int row, int k, int kp) {
    return (uint32_t)((row >> 3) * (kp >> 3) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// stores a 16-byte run (8 BF16 values of one row, k..k+7) into the canonical layout
__device__ __forceinline__ void tc_put16(unsigned char* base, int row, int k, int kp, uint4 v) {
    *(uint4*)(base + tc_off(row, k, kp)) = v;
}

// Persistent: each CTA loads W^T once, allocates its TMEM columns once, and
// walks over 128-row tiles (grid-stride); the mbarrier flips phase per tile.
// Wt is W transposed (N x K, K contiguous, leading dimension ldwt).
template <int EPI>
__global__ void __launch_bounds__(kTcThreads) k_gemm_tc(int M, int N, int K, const bf16* __restrict__ X, int ldx,
                                                       const bf16* __restrict__ Wt, int ldwt, GemmOut o, int* err) {
    extern __shared__ __align__(1024) unsigned char tc_sm[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ float s_out[kTcThreads / 32][32][17];  // per warp: 32 rows x 16 columns of the epilogue
    const int kp = (K + 15) & ~15, np = (N + 15) & ~15;
    unsigned char* sA = tc_sm;
    unsigned char* sB = tc_sm + (size_t)kTcM * kp * 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bf16 zero = __float2bfloat16(0.0f);
    const int kc = kp >> 3;  // 8-element runs per row
    const bool vec_x = (ldx & 7) == 0 && ((uintptr_t)X & 15) == 0 && K == kp;
    const bool vec_w = (ldwt & 7) == 0 && ((uintptr_t)Wt & 15) == 0 && K == kp;
    // W^T once: rows n < np, zero beyond N
    for (int e = tid; e < np * kc; e += kTcThreads) {
        const int n = e / kc, k = (e - n * kc) * 8;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (n < N) {
            if (vec_w) {
                v = *(const uint4*)(Wt + (size_t)n * ldwt + k);
            } else {
                bf16 t[8];
                for (int j = 0; j < 8; ++j) t[j] = k + j < K ? Wt[(size_t)n * ldwt + k + j] : zero;
                v = *(const uint4*)t;
            }
        }
        tc_put16(sB, n, k, kp, v);
    }
    const uint32_t ncols = np <= 32 ? 32u : (np <= 64 ? 64u : (np <= 128 ? 128u : 256u));
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_addr(&s_tmem)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_addr(&s_mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;
    const uint32_t a0 = tc_smem_addr(sA), b0 = tc_smem_addr(sB), sbo = (uint32_t)kc * 128u;
    const uint32_t idesc = tc_idesc_bf16(kTcM, np);
    const int n_tiles = (M + kTcM - 1) / kTcM;
    uint32_t phase = 0;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int m0 = tile * kTcM;
        // X tile: rows m0.., 16-byte runs when aligned
        for (int e = tid; e < kTcM * kc; e += kTcThreads) {
            const int r = e / kc, k = (e - r * kc) * 8, m = m0 + r;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (m < M) {
                if (vec_x) {
                    v = *(const uint4*)(X + (size_t)m * ldx + k);
                } else {
                    bf16 t[8];
                    for (int j = 0; j < 8; ++j) t[j] = k + j < K ? X[(size_t)m * ldx + k + j] : zero;
                    v = *(const uint4*)t;
                }
            }
            tc_put16(sA, r, k, kp, v);
        }
        // generic-proxy shared memory writes become visible to the tensor cores
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            for (int s = 0; s < kp / 16; ++s) {
                const uint64_t da = tc_desc(a0 + 256u * s, 128u, sbo), db = tc_desc(b0 + 256u * s, 128u, sbo);
                const uint32_t acc = s > 0 ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                tc_smem_addr(&s_mbar)));
        }
        // bounded wait for this tile's products (non-blocking polls)
        uint32_t done = 0;
        for (int i = 0; i < kTcSpinLimit && !done; ++i) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(tc_smem_addr(&s_mbar)), "r"(phase));
            if (!done && i >= 1024) __nanosleep(32);
        }
        phase ^= 1u;
        // a timed-out wait ends the kernel for the whole CTA (no further
        // products are issued on an mbarrier whose phase is unknown)
        if (__syncthreads_or(!done)) {
            if (tid == 0) atomicExch(err, 1);
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // epilogue: 16 accumulator columns at a time through shared memory so
        // that the global stores run along rows
        for (int c0 = 0; c0 < np; c0 += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int j = 0; j < 16; ++j) s_out[warp][lane][j] = __uint_as_float(r[j]);
            __syncwarp();
            // lane pair (row, 16 columns): half-warps cover two rows per step
            const int col = lane & 15, n = c0 + col;
            for (int rr = lane >> 4; rr < 32; rr += 2) {
                const int m = m0 + warp * 32 + rr;
                if (m < M && n < N) {
                    const float a = s_out[warp][rr][col];
                    const size_t i = (size_t)m * o.ld + n;
                    if (EPI == kEpiHidden) {
                        const float z = a + o.bias[n];
                        o.f[i] = z;
                        o.h[i] = __float2bfloat16(z > 0.0f ? z : 0.0f);
                    } else {
                        o.f[i] = a + o.bias[n];
                    }
                }
            }
            __syncwarp();
        }
        // all TMEM reads of this tile are done before the next tile's products
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

}  // namespace zema
