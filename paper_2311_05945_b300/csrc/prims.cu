// Exclusive scan and stable LSD radix sort (8-bit digits), written for the
// broad phase and the contact assembly.  Both are deterministic: no atomics
// decide an output position.
#include <string>
#include <vector>

#include "prims.cuh"

namespace zema {

long long& launch_counter() {
    static long long n = 0;
    return n;
}

// --- per-kernel timing (one selected kernel at a time) ---------------------
namespace {
struct Prof {
    std::string name;
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    size_t used = 0;
    double bytes = 0.0, pending = 0.0;
    long long launches = 0;
};
Prof& prof() {
    static Prof p;
    return p;
}
thread_local cudaStream_t g_stream = nullptr;
}  // namespace

void set_current_stream(cudaStream_t st) { g_stream = st; }
void alg_bytes_hint(double bytes) { prof().pending = bytes; }

void alg_bytes_add(const char* name, double bytes) {
    Prof& P = prof();
    if (P.on && P.name == name) P.bytes += bytes;
}

LaunchScope::LaunchScope(const char* name, bool count) : timed(false) {
    if (count) ++launch_counter();
    Prof& P = prof();
    if (!P.on) return;
    // match the kernel name, ignoring template arguments
    const char* a = name;
    const char* b = P.name.c_str();
    while (*a && *b && *a == *b) ++a, ++b;
    if (*b || (*a && *a != '<')) return;
    if (P.used == P.ev.size()) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        P.ev.push_back({e0, e1});
    }
    cudaEventRecord(P.ev[P.used].first, g_stream);
    timed = true;
}

LaunchScope::~LaunchScope() {
    if (!timed) return;
    Prof& P = prof();
    cudaEventRecord(P.ev[P.used].second, g_stream);
    ++P.used;
    ++P.launches;
    P.bytes += P.pending;
}

}  // namespace zema

extern "C" {
// Selects the kernel to time (NULL disables) and clears the totals.
int zema_profile_kernel(const char* name) {
    zema::Prof& P = zema::prof();
    P.on = name != nullptr;
    P.name = name ? name : "";
    P.used = 0;
    P.bytes = 0.0;
    P.pending = 0.0;
    P.launches = 0;
    return 0;
}

// Totals since zema_profile_kernel: summed event time of the selected
// kernel's launches, their count and their declared algorithmic bytes.
int zema_profile_read(double* ms_total, long long* launches, double* alg_bytes) {
    zema::Prof& P = zema::prof();
    double ms = 0.0;
    for (size_t i = 0; i < P.used; ++i) {
        cudaEventSynchronize(P.ev[i].second);
        float t = 0.f;
        if (cudaEventElapsedTime(&t, P.ev[i].first, P.ev[i].second) == cudaSuccess) ms += t;
    }
    if (ms_total) *ms_total = ms;
    if (launches) *launches = P.launches;
    if (alg_bytes) *alg_bytes = P.bytes;
    return 0;
}
}

namespace zema {

constexpr int SCAN_T = 256;
constexpr int SCAN_PER = 16;
constexpr int SCAN_TILE = SCAN_T * SCAN_PER;

// per-block exclusive scan of SCAN_TILE elements; block totals to sums; a
// single-block scan also writes the total to out[n] when `total` is set
__global__ void k_scan_block(const uint32_t* in, uint32_t* out, size_t n, uint32_t* sums, int total) {
    __shared__ uint32_t wsum[SCAN_T / 32];
    size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_PER;
    uint32_t v[SCAN_PER];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0u;
        s += v[i];
    }
    // inclusive warp scan of thread sums
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t ws = (lane < SCAN_T / 32) ? wsum[lane] : 0u;
        uint32_t wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < SCAN_T / 32) wsum[lane] = wi - ws;  // exclusive warp offsets
        if (lane == SCAN_T / 32 - 1) {
            sums[blockIdx.x] = wi;
            if (total) out[n] = wi;
        }
    }
    __syncthreads();
    uint32_t run = wsum[w] + inc - s;
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

// adds the scanned block offsets; the last block's thread 0 also writes the
// total to out[n] when `total` is set
__global__ void k_scan_add(uint32_t* out, size_t n, const uint32_t* offs, const uint32_t* sums, int total) {
    size_t i = (size_t)blockIdx.x * SCAN_TILE + threadIdx.x;
    uint32_t o = offs[blockIdx.x];
    for (int k = 0; k < SCAN_PER; ++k, i += SCAN_T)
        if (i < n) out[i] += o;
    if (total && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) out[n] = o + sums[blockIdx.x];
}

__global__ void k_set_total_zero(uint32_t* out) { out[0] = 0; }

// one CTA scans n <= SCAN1_T * SCAN1_PER elements (each thread a contiguous
// run of ceil(n / SCAN1_T)), out[n] = total: one launch instead of the
// three of the multi-block scan for mid-sized arrays
constexpr int SCAN1_T = 1024;
constexpr int SCAN1_PER = 32;
__global__ void __launch_bounds__(SCAN1_T) k_scan_single(const uint32_t* in, uint32_t* out, int n) {
    __shared__ uint32_t wsum[SCAN1_T / 32];
    const int per = (n + SCAN1_T - 1) / SCAN1_T;
    const int b = threadIdx.x * per, e = min(n, b + per);
    uint32_t s = 0;
    for (int i = b; i < e; ++i) s += in[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        const uint32_t ws = wsum[lane];
        uint32_t wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        wsum[lane] = wi - ws;  // exclusive warp offsets
        if (lane == 31) out[n] = wi;
    }
    __syncthreads();
    uint32_t run = wsum[w] + inc - s;
    for (int i = b; i < e; ++i) {
        const uint32_t v = in[i];
        out[i] = run;
        run += v;
    }
}

size_t scan_tmp_size(size_t n) {
    size_t total = 0;
    size_t m = n;
    while (m > SCAN_TILE) {
        size_t nb = (m + SCAN_TILE - 1) / SCAN_TILE;
        total += 2 * nb + 2;
        m = nb;
    }
    return total + 2 * SCAN_TILE + 8;
}

static void scan_rec(const uint32_t* in, uint32_t* out, size_t n, uint32_t* tmp, int total, cudaStream_t st) {
    size_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    uint32_t* sums = tmp;
    uint32_t* soff = tmp + nb + 1;
    ZL(k_scan_block, (unsigned)nb, SCAN_T, 0, st)(in, out, n, sums, total && nb == 1);
    ZLAUNCH();
    if (nb > 1) {
        scan_rec(sums, soff, nb, tmp + 2 * nb + 2, 0, st);
        ZL(k_scan_add, (unsigned)nb, SCAN_T, 0, st)(out, n, soff, sums, total);
        ZLAUNCH();
    }
}

// out[0..n) = exclusive scan of in, out[n] = total
void exclusive_scan(const uint32_t* in, uint32_t* out, size_t n, uint32_t* tmp, cudaStream_t st) {
    if (n == 0) {
        ZL(k_set_total_zero, 1, 1, 0, st)(out);
        ZLAUNCH();
        return;
    }
    if (n > SCAN_TILE && n <= (size_t)SCAN1_T * SCAN1_PER) {
        ZL(k_scan_single, 1, SCAN1_T, 0, st)(in, out, (int)n);
        ZLAUNCH();
        return;
    }
    scan_rec(in, out, n, tmp, 1, st);
}

// ---------------------------------------------------------------------------
// Radix sort
// ---------------------------------------------------------------------------
constexpr int RS_T = 256;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_T * RS_ROUNDS;
constexpr int RS_WARPS = RS_T / 32;

__global__ void k_rs_hist(const uint64_t* keys, size_t n, int shift, uint32_t* hist, int ntiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    size_t base = (size_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        size_t i = base + (size_t)r * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_rs_scatter(const uint64_t* keys, const uint32_t* vals, uint64_t* ko, uint32_t* vo, size_t n,
                             int shift, const uint32_t* offs, int ntiles) {
    __shared__ uint32_t wc[RS_WARPS][256];
    __shared__ uint32_t run[256];
    __shared__ uint32_t gbase[256];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    run[threadIdx.x] = 0;
    gbase[threadIdx.x] = offs[(size_t)threadIdx.x * ntiles + blockIdx.x];
    for (int k = 0; k < RS_WARPS; ++k) wc[k][threadIdx.x] = 0;
    __syncthreads();
    size_t base = (size_t)blockIdx.x * RS_TILE;
    unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        size_t i = base + (size_t)r * RS_T + threadIdx.x;
        bool valid = i < n;
        uint64_t key = valid ? keys[i] : 0ull;
        uint32_t val = valid ? vals[i] : 0u;
        unsigned dig = valid ? (unsigned)((key >> shift) & 255u) : 256u + lane;
        unsigned peers = __match_any_sync(0xffffffffu, dig);
        unsigned rank = __popc(peers & lt);
        if (valid && rank == 0) wc[w][dig] = __popc(peers);
        __syncthreads();
        {
            int d = threadIdx.x;
            uint32_t acc = run[d];
            for (int k = 0; k < RS_WARPS; ++k) {
                uint32_t t = wc[k][d];
                wc[k][d] = acc;
                acc += t;
            }
            run[d] = acc;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = gbase[dig] + wc[w][dig] + rank;
            ko[pos] = key;
            vo[pos] = val;
        }
        __syncthreads();
        for (int k = 0; k < RS_WARPS; ++k) wc[k][threadIdx.x] = 0;
        __syncthreads();
    }
}

size_t radix_tmp_size(size_t n) {
    size_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    size_t h = 256 * ntiles;
    return 2 * h + 2 + scan_tmp_size(h);
}

void radix_sort(uint64_t* keys, uint32_t* vals, uint64_t* k2, uint32_t* v2, size_t n, int bits, uint32_t* tmp,
                cudaStream_t st) {
    if (n <= 1) return;
    int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    size_t h = 256 * (size_t)ntiles;
    uint32_t* hist = tmp;
    uint32_t* offs = tmp + h + 1;
    uint32_t* stmp = tmp + 2 * h + 2;
    int passes = (bits + 7) / 8;
    uint64_t *ka = keys, *kb = k2;
    uint32_t *va = vals, *vb = v2;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        ZL(k_rs_hist, ntiles, RS_T, 0, st)(ka, n, shift, hist, ntiles);
        ZLAUNCH();
        exclusive_scan(hist, offs, h, stmp, st);
        ZL(k_rs_scatter, ntiles, RS_T, 0, st)(ka, va, kb, vb, n, shift, offs, ntiles);
        ZLAUNCH();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        ZCHECK(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
        ZCHECK(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    }
}

}  // namespace zema
