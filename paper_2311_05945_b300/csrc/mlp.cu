// Tensor-core MLP: BF16 operands, FP32 accumulation, deterministic training.
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "mlp.cuh"
#include "mlp_tc.cuh"

namespace zema {

constexpr int GB_M = 64, GB_N = 64, GB_K = 32, GB_T = 128, GB_PAD = 8;

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld_pair(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// C = op(A) op(B), A(m, k) = TA ? A[k lda + m] : A[m lda + k],
// B(k, n) = TB ? B[n ldb + k] : B[k ldb + n].  CTA tile 64 x 64 x 32, four
// warps of 32 x 32 (2 x 4 mma tiles of 16 x 8).  blockIdx.z splits K into
// chunks of kps (kEpiStore writes one partial per split).
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(GB_T) k_gemm_bf16(int M, int N, int K, const bf16* __restrict__ A, int lda,
                                                   const bf16* __restrict__ B, int ldb, GemmOut o, int kps) {
    __shared__ __align__(16) bf16 As[GB_M][GB_K + GB_PAD];
    __shared__ __align__(16) bf16 Bs[GB_N][GB_K + GB_PAD];  // n-major: B(k, n) at Bs[n][k]
    const int m0 = blockIdx.x * GB_M, n0 = blockIdx.y * GB_N;
    const int k_begin = blockIdx.z * kps, k_end = min(K, k_begin + kps);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    const bf16 zero = __float2bfloat16(0.0f);
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;
    for (int k0 = k_begin; k0 < k_end; k0 += GB_K) {
        // tiles from global memory, consecutive threads along the contiguous dimension
        for (int e = tid; e < GB_M * GB_K; e += GB_T) {
            const int r = TA ? e % GB_M : e / GB_K, c = TA ? e / GB_M : e % GB_K;
            const int m = m0 + r, k = k0 + c;
            bf16 v = zero;
            if (m < M && k < k_end) v = TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
            As[r][c] = v;
        }
        for (int e = tid; e < GB_N * GB_K; e += GB_T) {
            const int r = TB ? e / GB_K : e % GB_N, c = TB ? e % GB_K : e / GB_N;
            const int n = n0 + r, k = k0 + c;
            bf16 v = zero;
            if (n < N && k < k_end) v = TB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
            Bs[r][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GB_K; ks += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r = wm + mt * 16 + g;
                af[mt][0] = ld_pair(&As[r][ks + 2 * t]);
                af[mt][1] = ld_pair(&As[r + 8][ks + 2 * t]);
                af[mt][2] = ld_pair(&As[r][ks + 2 * t + 8]);
                af[mt][3] = ld_pair(&As[r + 8][ks + 2 * t + 8]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int cidx = wn + nt * 8 + g;
                bfr[nt][0] = ld_pair(&Bs[cidx][ks + 2 * t]);
                bfr[nt][1] = ld_pair(&Bs[cidx][ks + 2 * t + 8]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
                    mma_bf16_16816(acc[mt][nt], af[mt][0], af[mt][1], af[mt][2], af[mt][3], bfr[nt][0], bfr[nt][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + wm + mt * 16 + g + (q >> 1) * 8, n = n0 + wn + nt * 8 + 2 * t + (q & 1);
                if (m >= M || n >= N) continue;
                const float a = acc[mt][nt][q];
                const size_t i = (size_t)m * o.ld + n;
                if (EPI == kEpiStore) {
                    o.f[(size_t)blockIdx.z * M * o.ld + i] = a;
                } else if (EPI == kEpiHidden) {
                    const float z = a + o.bias[n];
                    o.f[i] = z;
                    o.h[i] = __float2bfloat16(z > 0.0f ? z : 0.0f);
                } else if (EPI == kEpiOut) {
                    o.f[i] = a + o.bias[n];
                } else {
                    o.h[i] = __float2bfloat16(o.z_in[i] > 0.0f ? a : 0.0f);
                }
            }
}

// out[i] (+)= sum over splits s of part[s][i], in split order
__global__ void k_sum_splits(const float* part, int splits, size_t n, float* out) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.0f;
    for (int k = 0; k < splits; ++k) s += part[(size_t)k * n + i];
    out[i] = s;
}

__global__ void k_f32_to_bf16(const float* a, bf16* b, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16(a[i]);
}

// W (k x n, row-major) -> W^T (n x k, row-major) in BF16
__global__ void k_transpose_bf16(const float* w, int k, int n, bf16* wt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k * n) return;
    const int r = i / n, c = i - r * n;
    wt[(size_t)c * k + r] = __float2bfloat16(w[i]);
}

__global__ void k_fill_bf16(bf16* b, size_t n, float v) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16(v);
}

// MSE: per-block partial of sum (y - t)^2, and dy = 2 (y - t) / (n out)
__global__ void k_mse(const float* y, const float* t, size_t n, float scale, bf16* dy, float* part) {
    __shared__ double sh[32];
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (i < n) {
        const float d = y[i] - t[i];
        dy[i] = __float2bfloat16(scale * d);
        e = (double)d * d;
    }
    double s = block_sum<256>(e, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = (float)s;
}

__global__ void k_adamw(float* th, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2,
                        float eps, float wd, float c1, float c2, bf16* th_bf) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = (mi * c1) / (sqrtf(vi * c2) + eps) + wd * th[i];
    const float w = th[i] - lr * upd;
    th[i] = w;
    th_bf[i] = __float2bfloat16(w);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

uint64_t sm64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// launches the product; returns the number of K splits used
template <bool TA, bool TB, int EPI>
int gemm(cudaStream_t st, int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb, GemmOut o,
         int splits = 1) {
    if (M <= 0 || N <= 0) return 0;
    int kps = K;
    if (splits > 1) {
        kps = (K + splits - 1) / splits;
        kps = (kps + GB_K - 1) / GB_K * GB_K;
        splits = std::max(1, (K + kps - 1) / kps);
    }
    dim3 grid(div_up(M, GB_M), div_up(N, GB_N), splits);
    ZL((k_gemm_bf16<TA, TB, EPI>), grid, GB_T, 0, st)(M, N, K, A, lda, B, ldb, o, kps);
    ZLAUNCH();
    return splits;
}

// forward product on tcgen05 (K <= 128, N <= 256): persistent CTAs, two per SM
template <int EPI>
void gemm_tc(cudaStream_t st, int M, int N, int K, const bf16* X, int ldx, const bf16* Wt, int ldwt, GemmOut o,
             int* err) {
    if (M <= 0 || N <= 0) return;
    const int kp = (K + 15) & ~15, np = (N + 15) & ~15;
    const size_t smem = (size_t)(kTcM + np) * kp * 2;
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        ZCHECK(cudaGetDevice(&dev));
        ZCHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        ZCHECK(cudaFuncSetAttribute(k_gemm_tc<kEpiHidden>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
        ZCHECK(cudaFuncSetAttribute(k_gemm_tc<kEpiOut>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    }
    const int grid = std::min(div_up(M, kTcM), 2 * nsm);
    ZL(k_gemm_tc<EPI>, grid, kTcThreads, smem, st)(M, N, K, X, ldx, Wt, ldwt, o, err);
    ZLAUNCH();
}

bool tc_fits(int K, int N) { return K <= 128 && N <= 256; }

// splits of a K-reduction of length K so that a 1 x 2 (or 2 x 2) tile grid
// still fills the GPU
int splits_for(int64_t K) { return (int)std::min<int64_t>(256, std::max<int64_t>(1, K / 512)); }

}  // namespace

Mlp::Mlp(const std::vector<int>& d, uint64_t seed, cudaStream_t s) : dims(d), st(s) {
    A.stream = s;
    const int L = layers();
    size_t off = 0;
    for (int l = 0; l < L; ++l) {
        w_off.push_back(off);
        off += (size_t)dims[l] * dims[l + 1];
        b_off.push_back(off);
        off += dims[l + 1];
    }
    n_params = off;
    theta.ensure(&A, n_params);
    grad.ensure(&A, n_params);
    m.ensure(&A, n_params);
    v.ensure(&A, n_params);
    theta_bf.ensure(&A, n_params);
    theta_t.ensure(&A, n_params);
    tc_err.ensure(&A, 1);
    ZCHECK(cudaMemsetAsync(tc_err.p, 0, sizeof(int), st));
    // He-uniform weights from SplitMix64 (last layer scaled by 0.1), zero biases
    std::vector<float> init(n_params, 0.0f);
    uint64_t rs = seed;
    for (int l = 0; l < L; ++l) {
        const double a = std::sqrt(6.0 / dims[l]) * (l == L - 1 ? 0.1 : 1.0);
        for (size_t i = 0; i < (size_t)dims[l] * dims[l + 1]; ++i) {
            const double u = (double)(sm64(rs) >> 11) * (1.0 / 9007199254740992.0);
            init[w_off[l] + i] = (float)((2.0 * u - 1.0) * a);
        }
    }
    ZCHECK(cudaMemcpyAsync(theta.p, init.data(), n_params * sizeof(float), cudaMemcpyHostToDevice, st));
    ZCHECK(cudaMemsetAsync(m.p, 0, n_params * sizeof(float), st));
    ZCHECK(cudaMemsetAsync(v.p, 0, n_params * sizeof(float), st));
    refresh_bf16();
    for (int l = 0; l + 1 < L; ++l) {
        z.push_back(new DBuf<float>());
        h.push_back(new DBuf<bf16>());
    }
    ZCHECK(cudaStreamSynchronize(st));
}

Mlp::~Mlp() {
    for (auto* p : z) delete p;
    for (auto* p : h) delete p;
}

void Mlp::refresh_bf16() {
    ZL(k_f32_to_bf16, div_up(n_params, 256), 256, 0, st)(theta.p, theta_bf.p, n_params);
    refresh_t();
    ZLAUNCH();
}

// the transposed BF16 weights read by the tcgen05 products
void Mlp::refresh_t() {
    for (int l = 0; l < layers(); ++l)
        ZL(k_transpose_bf16, div_up(dims[l] * dims[l + 1], 256), 256, 0, st)(theta.p + w_off[l], dims[l], dims[l + 1],
                                                                              theta_t.p + w_off[l]);
    ZLAUNCH();
}

void Mlp::ensure_rows(int64_t n) {
    if (n <= cap_rows) return;
    const int L = layers();
    int wmax = 0;
    for (int w : dims) wmax = std::max(wmax, w);
    for (int l = 0; l + 1 < L; ++l) {
        z[l]->ensure(&A, (size_t)n * dims[l + 1]);
        h[l]->ensure(&A, (size_t)n * dims[l + 1]);
    }
    xb.ensure(&A, (size_t)n * dims[0]);
    y.ensure(&A, (size_t)n * dims[L]);
    dy.ensure(&A, (size_t)n * dims[L]);
    dg0.ensure(&A, (size_t)n * wmax);
    dg1.ensure(&A, (size_t)n * wmax);
    ones.ensure(&A, (size_t)n);
    ZL(k_fill_bf16, div_up(n, 256), 256, 0, st)(ones.p, (size_t)n, 1.0f);
    ZLAUNCH();
    loss_part.ensure(&A, (size_t)div_up((size_t)n * dims[L], 256) + 1);
    part.ensure(&A, (size_t)256 * wmax * wmax);
    cap_rows = n;
}

void Mlp::forward(const float* x, int64_t n, float* y_out) {
    ensure_rows(n);
    const int L = layers();
    ZL(k_f32_to_bf16, div_up((size_t)n * dims[0], 256), 256, 0, st)(x, xb.p, (size_t)n * dims[0]);
    ZLAUNCH();
    const bf16* in = xb.p;
    for (int l = 0; l < L; ++l) {
        const int K = dims[l], N = dims[l + 1];
        GemmOut o{};
        o.bias = theta.p + b_off[l];
        o.ld = N;
        const bf16* W = theta_bf.p + w_off[l];
        const bool tc = use_tc && tc_fits(K, N);
        if (l + 1 < L) {
            o.f = z[l]->p;
            o.h = h[l]->p;
            if (tc)
                gemm_tc<kEpiHidden>(st, (int)n, N, K, in, K, theta_t.p + w_off[l], K, o, tc_err.p);
            else
                gemm<false, false, kEpiHidden>(st, (int)n, N, K, in, K, W, N, o);
            in = h[l]->p;
        } else {
            o.f = y_out ? y_out : y.p;
            if (tc)
                gemm_tc<kEpiOut>(st, (int)n, N, K, in, K, theta_t.p + w_off[l], K, o, tc_err.p);
            else
                gemm<false, false, kEpiOut>(st, (int)n, N, K, in, K, W, N, o);
        }
    }
}

double Mlp::backward(const float* x, const float* t, int64_t n) {
    const int L = layers();
    forward(x, n, nullptr);
    const size_t ny = (size_t)n * dims[L];
    const int nb = div_up(ny, 256);
    ZL(k_mse, nb, 256, 0, st)(y.p, t, ny, 2.0f / (float)ny, dy.p, loss_part.p);
    ZLAUNCH();
    const bf16* dz = dy.p;
    bf16* bufs[2] = {dg0.p, dg1.p};
    for (int l = L - 1; l >= 0; --l) {
        const int K = dims[l], N = dims[l + 1];
        const bf16* hin = l == 0 ? xb.p : h[l - 1]->p;
        const int sp = splits_for(n);
        // dW_l = H_{l-1}^T dZ_l  (K x N), split over the rows, summed in order
        GemmOut o{};
        o.f = part.p;
        o.ld = N;
        int used = gemm<true, false, kEpiStore>(st, K, N, (int)n, hin, K, dz, N, o, sp);
        ZL(k_sum_splits, div_up((size_t)K * N, 256), 256, 0, st)(part.p, used, (size_t)K * N, grad.p + w_off[l]);
        // db_l = 1^T dZ_l
        used = gemm<false, false, kEpiStore>(st, 1, N, (int)n, ones.p, (int)n, dz, N, o, sp);
        ZL(k_sum_splits, div_up((size_t)N, 256), 256, 0, st)(part.p, used, (size_t)N, grad.p + b_off[l]);
        ZLAUNCH();
        if (l > 0) {
            // dZ_{l-1} = (dZ_l W_l^T) * relu'(Z_{l-1})
            GemmOut ob{};
            ob.h = bufs[l & 1];
            ob.z_in = z[l - 1]->p;
            ob.ld = K;
            gemm<false, true, kEpiReluBack>(st, (int)n, K, N, dz, N, theta_bf.p + w_off[l], N, ob);
            dz = bufs[l & 1];
        }
    }
    std::vector<float> lp(nb);
    ZCHECK(cudaMemcpyAsync(lp.data(), loss_part.p, nb * sizeof(float), cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaStreamSynchronize(st));
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += lp[i];
    return s / (double)ny;
}

void Mlp::adamw(float lr, float b1, float b2, float eps, float wd) {
    ++step;
    const float c1 = 1.0f / (1.0f - std::pow(b1, (float)step));
    const float c2 = 1.0f / (1.0f - std::pow(b2, (float)step));
    ZL(k_adamw, div_up(n_params, 256), 256, 0, st)(theta.p, grad.p, m.p, v.p, n_params, lr, b1, b2, eps, wd, c1, c2,
                                                  theta_bf.p);
    ZLAUNCH();
    if (use_tc) refresh_t();
}

}  // namespace zema

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
struct zema_mlp {
    zema::Mlp* net = nullptr;
};

using zema::ZemaError;

static zema_status mlp_status(const ZemaError& e) { return (zema_status)e.status; }

extern "C" zema_status zema_mlp_create(const int32_t* dims, int32_t n_layers, uint64_t seed, void* stream,
                                       zema_mlp** out) {
    if (!dims || !out || n_layers < 1 || n_layers > 16) return ZEMA_ERR_INVALID_ARG;
    for (int l = 0; l <= n_layers; ++l)
        if (dims[l] < 1 || dims[l] > 4096) return ZEMA_ERR_INVALID_ARG;
    zema_mlp* m = new (std::nothrow) zema_mlp();
    if (!m) return ZEMA_ERR_OOM;
    try {
        m->net = new zema::Mlp(std::vector<int>(dims, dims + n_layers + 1), seed, (cudaStream_t)stream);
    } catch (const ZemaError& e) {
        delete m;
        return mlp_status(e);
    } catch (...) {
        delete m;
        return ZEMA_ERR_OOM;
    }
    *out = m;
    return ZEMA_OK;
}

extern "C" void zema_mlp_destroy(zema_mlp* m) {
    if (!m) return;
    delete m->net;
    delete m;
}

extern "C" zema_status zema_mlp_n_params(const zema_mlp* m, int64_t* n) {
    if (!m || !n) return ZEMA_ERR_INVALID_ARG;
    *n = (int64_t)m->net->n_params;
    return ZEMA_OK;
}

extern "C" zema_status zema_mlp_get_params(const zema_mlp* m, float* out, int64_t cap) {
    if (!m || !out || cap < (int64_t)m->net->n_params) return ZEMA_ERR_INVALID_ARG;
    try {
        ZCHECK(cudaMemcpyAsync(out, m->net->theta.p, m->net->n_params * sizeof(float), cudaMemcpyDeviceToHost,
                               m->net->st));
        ZCHECK(cudaStreamSynchronize(m->net->st));
        return ZEMA_OK;
    } catch (const ZemaError& e) {
        return mlp_status(e);
    }
}

extern "C" zema_status zema_mlp_set_params(zema_mlp* m, const float* in, int64_t n) {
    if (!m || !in || n != (int64_t)m->net->n_params) return ZEMA_ERR_INVALID_ARG;
    try {
        ZCHECK(cudaMemcpyAsync(m->net->theta.p, in, n * sizeof(float), cudaMemcpyHostToDevice, m->net->st));
        m->net->refresh_bf16();
        ZCHECK(cudaStreamSynchronize(m->net->st));
        return ZEMA_OK;
    } catch (const ZemaError& e) {
        return mlp_status(e);
    }
}

static void check_tc(zema::Mlp* net) {
    int e = 0;
    ZCHECK(cudaMemcpyAsync(&e, net->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, net->st));
    ZCHECK(cudaStreamSynchronize(net->st));
    if (e) throw ZemaError{ZEMA_ERR_CUDA, "tensor-core product did not complete"};
}

extern "C" zema_status zema_mlp_set_kernel(zema_mlp* m, int32_t kind) {
    if (!m || kind < 0 || kind > 1) return ZEMA_ERR_INVALID_ARG;
    try {
        m->net->use_tc = kind == 0 ? 1 : 0;
        if (m->net->use_tc) m->net->refresh_t();
        return ZEMA_OK;
    } catch (const ZemaError& e) {
        return mlp_status(e);
    }
}

extern "C" zema_status zema_mlp_forward(zema_mlp* m, const float* x, int64_t n, float* y) {
    if (!m || n < 0 || (n && (!x || !y))) return ZEMA_ERR_INVALID_ARG;
    if (n == 0) return ZEMA_OK;
    try {
        m->net->forward(x, n, y);
        check_tc(m->net);
        return ZEMA_OK;
    } catch (const ZemaError& e) {
        return mlp_status(e);
    }
}

extern "C" zema_status zema_mlp_gradient(zema_mlp* m, const float* x, const float* t, int64_t n, float* grad,
                                         int64_t cap, double* loss) {
    if (!m || !x || !t || n < 1 || !grad || cap < (int64_t)m->net->n_params) return ZEMA_ERR_INVALID_ARG;
    try {
        double l = m->net->backward(x, t, n);
        check_tc(m->net);
        ZCHECK(cudaMemcpyAsync(grad, m->net->grad.p, m->net->n_params * sizeof(float), cudaMemcpyDeviceToHost,
                               m->net->st));
        ZCHECK(cudaStreamSynchronize(m->net->st));
        if (loss) *loss = l;
        return ZEMA_OK;
    } catch (const ZemaError& e) {
        return mlp_status(e);
    }
}

extern "C" zema_status zema_mlp_train_step(zema_mlp* m, const float* x, const float* t, int64_t n, float lr,
                                           float beta1, float beta2, float eps, float weight_decay, double* loss) {
    if (!m || !x || !t || n < 1 || !(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1))
        return ZEMA_ERR_INVALID_ARG;
    try {
        double l = m->net->backward(x, t, n);
        check_tc(m->net);
        m->net->adamw(lr, beta1, beta2, eps, weight_decay);
        if (loss) *loss = l;
        return ZEMA_OK;
    } catch (const ZemaError& e) {
        return mlp_status(e);
    }
}
