// Device primitives: device buffers, exclusive scan, stable radix sort.
#pragma once
#include <vector>

#include "../../include/zema.h"
#include "common.cuh"

namespace zema {

// Allocator used by every device buffer of a scene.
struct Allocator {
    zema_alloc_fn fa = nullptr;
    zema_free_fn ff = nullptr;
    void* ctx = nullptr;
    cudaStream_t stream = nullptr;
    size_t bytes_live = 0;
    void* get(size_t bytes) {
        if (bytes == 0) bytes = 16;
        void* p = nullptr;
        if (fa) {
            p = fa(bytes, (void*)stream, ctx);
            if (!p) throw ZemaError{2, "device allocation failed"};
        } else {
            cudaError_t e = cudaMalloc(&p, bytes);
            // out of memory is ZEMA_ERR_OOM; any other failure (no device, a
            // lost context) is ZEMA_ERR_CUDA
            if (e != cudaSuccess)
                throw ZemaError{e == cudaErrorMemoryAllocation ? 2 : 3,
                                std::string("cudaMalloc: ") + cudaGetErrorString(e)};
        }
        bytes_live += bytes;
        return p;
    }
    void put(void* p, size_t bytes) {
        if (!p) return;
        bytes_live -= bytes;
        if (ff)
            ff(p, (void*)stream, ctx);
        else
            cudaFree(p);
    }
};

template <class T>
struct DBuf {
    T* p = nullptr;
    size_t cap = 0;
    Allocator* A = nullptr;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p && A) A->put(p, cap * sizeof(T));
        p = nullptr;
        cap = 0;
    }
    // capacity for n elements; contents are not preserved when it grows
    T* ensure(Allocator* a, size_t n) {
        A = a;
        if (n <= cap && p) return p;
        release();
        size_t c = n < 64 ? 64 : n + n / 4;
        p = (T*)A->get(c * sizeof(T));
        cap = c;
        return p;
    }
    void upload(Allocator* a, const std::vector<T>& v) {
        ensure(a, v.size());
        if (!v.empty())
            ZCHECK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, a->stream));
    }
};

// out[0..n] = exclusive prefix sums of in[0..n-1]; out[n] = total.
// tmp must hold scan_tmp_size(n) uint32.
size_t scan_tmp_size(size_t n);
void exclusive_scan(const uint32_t* in, uint32_t* out, size_t n, uint32_t* tmp, cudaStream_t st);

// Stable LSD radix sort of (keys, vals) on the low `bits` bits of the keys.
// Results end in keys/vals; k2/v2 are scratch of the same size; tmp holds
// radix_tmp_size(n) uint32.
size_t radix_tmp_size(size_t n);
void radix_sort(uint64_t* keys, uint32_t* vals, uint64_t* k2, uint32_t* v2, size_t n, int bits, uint32_t* tmp,
                cudaStream_t st);

}  // namespace zema
