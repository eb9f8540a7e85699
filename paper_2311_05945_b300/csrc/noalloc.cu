// Broad phase for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc while they run the contact query: code
// that records work into a CUDA stream capture (where allocation calls are
// not allowed), runtimes that hand out all device memory up front from a
// fixed pool, or real-time loops that forbid allocator calls for latency.
// zema_candidates_raw_noalloc serves them: it takes device buffers for its
// inputs and outputs and keeps every scratch buffer of the broad phase in one
// file-scope device array of fixed size, so no call allocates.
#include <map>
#include <mutex>

#include "broadphase.cuh"

namespace {

// 64 MiB of scratch: held by every GPU that loads the library, until exit.
constexpr size_t kNoallocScratchBytes = 64ull << 20;
// largest accepted problem: surface vertices + edges + triangles
constexpr int64_t kNoallocMaxPrims = 1 << 16;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// per device: the device address of g_noalloc_scratch (host code only sees a
// host-side stand-in under that name)
std::mutex g_mu;
std::map<int, void*> g_addr;

struct Bump {
    char* base;
    size_t used, cap;
};

void* bump_alloc(size_t bytes, void*, void* ctx) {
    Bump* b = (Bump*)ctx;
    size_t off = (b->used + 255) & ~(size_t)255;
    if (off + bytes > b->cap) return nullptr;  // surfaces as ZEMA_ERR_OOM
    b->used = off + bytes;
    return b->base + off;
}

void bump_free(void*, void*, void*) {}

__global__ void k_noalloc_sv_env(const int* sv_body, const int* b_env, int n, int* sv_env) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) sv_env[i] = b_env[sv_body[i]];
}

}  // namespace

extern "C" zema_status zema_candidates_raw_noalloc(int64_t nsv, const double* pos0, const double* pos1,
                                                   const int32_t* sv_body, int64_t nb, const int32_t* b_class,
                                                   const int32_t* b_env, int64_t ne, const int32_t* edges,
                                                   int64_t nt, const int32_t* tris, double inflate, double cell_size,
                                                   int64_t cap, int32_t* pt_out, int32_t* ee_out, int64_t* n_out,
                                                   void* stream) {
    if (nsv < 0 || nb < 1 || ne < 0 || nt < 0 || !pos0 || !sv_body || !b_class || !b_env || !n_out || !pt_out ||
        !ee_out || cap < 0 || !(inflate >= 0) || !(cell_size > 0))
        return ZEMA_ERR_INVALID_ARG;
    if (nsv + ne + nt > kNoallocMaxPrims) return ZEMA_ERR_INVALID_ARG;  // beyond the fixed scratch's limit
    if ((ne && !edges) || (nt && !tris)) return ZEMA_ERR_INVALID_ARG;
    using namespace zema;
    cudaStream_t st = (cudaStream_t)stream;
    try {
        set_current_stream(st);
        int dev = 0;
        ZCHECK(cudaGetDevice(&dev));
        void* base = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_mu);
            auto it = g_addr.find(dev);
            if (it == g_addr.end()) {
                // first call on this device: resolve the array's device address
                // (do this before any stream capture)
                ZCHECK(cudaGetSymbolAddress(&base, g_noalloc_scratch));
                g_addr[dev] = base;
            } else {
                base = it->second;
            }
        }
        Bump bump{(char*)base, 0, kNoallocScratchBytes};
        Allocator A;
        A.fa = bump_alloc;
        A.ff = bump_free;
        A.ctx = &bump;
        A.stream = st;
        // sv_env from the body envs, in the fixed scratch
        int* sve = (int*)A.get(((size_t)nsv + 1) * sizeof(int));
        if (nsv) ZL(k_noalloc_sv_env, div_up(nsv, 256), 256, 0, st)(sv_body, b_env, (int)nsv, sve);
        ZLAUNCH();
        BPView v;
        v.nsv = (int)nsv;
        v.ne = (int)ne;
        v.nt = (int)nt;
        v.X0 = pos0;
        v.X1 = pos1;
        v.sv_body = sv_body;
        v.body_class = b_class;
        v.sv_env = sve;
        v.edges = (const int2*)edges;
        v.tris = (const int3*)tris;
        v.infl = inflate;
        v.inv_cell = 1.0 / cell_size;
        static uint32_t host_counts[16];  // pageable: no pinned allocation
        BroadPhase bp;
        bp.h_counts = host_counts;
        zema_status status = ZEMA_OK;
        try {
            bp.run(&A, v, st);
            n_out[0] = bp.n_pt;
            n_out[1] = bp.n_ee;
            size_t mp = std::min<size_t>(bp.n_pt, (size_t)cap), me = std::min<size_t>(bp.n_ee, (size_t)cap);
            if (mp) ZCHECK(cudaMemcpyAsync(pt_out, bp.pt.p, mp * sizeof(int2), cudaMemcpyDeviceToDevice, st));
            if (me) ZCHECK(cudaMemcpyAsync(ee_out, bp.ee.p, me * sizeof(int2), cudaMemcpyDeviceToDevice, st));
            ZCHECK(cudaStreamSynchronize(st));
        } catch (const ZemaError& e) {
            status = (zema_status)e.status;
        }
        bp.h_counts = nullptr;  // static storage: not for cudaFreeHost
        return status;
    } catch (const ZemaError& e) {
        return (zema_status)e.status;
    }
}
