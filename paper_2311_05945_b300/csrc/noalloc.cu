// Broad phase for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc while they run the contact query:
// runtimes that hand out all device memory up front from a fixed pool, or
// real-time loops that forbid allocator calls for latency.
// zema_candidates_raw_noalloc serves them: it takes device buffers for its
// inputs and outputs and keeps every scratch buffer of the broad phase in one
// file-scope device array of fixed size, so no call allocates.  The call is
// not for stream capture: it synchronises its stream and reads counts back to
// the host partway through, to size the following launches.
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

// Checks the caller's device index arrays before any kernel indexes with
// them: body ids in [0, nb), body classes in [0, 3], envs >= 0, edge and
// triangle vertices in [0, nsv).  A bad entry sets *bad (no access is made
// through it).
__global__ void k_noalloc_check(const int* sv_body, int nsv, const int* b_class, const int* b_env, int nb,
                                const int* edges, int ne, const int* tris, int nt, int* bad) {
    const long long n = (long long)nsv + nb + 2ll * ne + 3ll * nt;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        bool ok;
        if (i < nsv) {
            ok = sv_body[i] >= 0 && sv_body[i] < nb;
        } else if (i < nsv + nb) {
            const long long b = i - nsv;
            ok = b_class[b] >= 0 && b_class[b] <= 3 && b_env[b] >= 0;
        } else {
            const long long k = i - nsv - nb;
            const int v = k < 2ll * ne ? edges[k] : tris[k - 2ll * ne];
            ok = v >= 0 && v < nsv;
        }
        if (!ok) *bad = 1;
    }
}

// env of every surface vertex from its body (ids checked above)
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
        // the caller's index arrays, checked on the device before use
        int* bad = (int*)A.get(sizeof(int));
        ZCHECK(cudaMemsetAsync(bad, 0, sizeof(int), st));
        ZL(k_noalloc_check, 148, 256, 0, st)(sv_body, (int)nsv, b_class, b_env, (int)nb, edges, (int)ne, tris,
                                             (int)nt, bad);
        ZLAUNCH();
        int bad_h = 0;
        ZCHECK(cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        ZCHECK(cudaStreamSynchronize(st));
        if (bad_h) return ZEMA_ERR_INVALID_ARG;
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
        uint32_t host_counts[16];  // this call's own (pageable: no pinned allocation)
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
            // kernels queued before the failure still use the array: let them
            // finish before another call may reuse it
            cudaStreamSynchronize(st);
        }
        bp.h_counts = nullptr;  // stack storage: not for cudaFreeHost
        return status;
    } catch (const ZemaError& e) {
        return (zema_status)e.status;
    }
}
