// Spatial-hash broad phase over surface point-triangle and edge-edge pairs
// (the paper's "DCD" stage, Table I, done with a uniform grid instead of a
// BVH).  Produces every valid pair whose axis-aligned boxes, inflated by
// `infl` per side (and swept over X0 -> X1 when X1 is given), overlap.
#pragma once
#include "prims.cuh"

namespace zema {

struct BPView {
    int nsv, ne, nt;
    const double* X0;
    const double* X1;  // nullable: swept boxes over X0 -> X1
    const int* sv_body;
    const int* body_class;  // 0 soft, 1 affine dynamic, 2 fixed, 3 kinematic
    const int* sv_env;
    const int2* edges;
    const int3* tris;
    double infl;
    double inv_cell;
    const int* env_skip = nullptr;  // nullable, per env: 1 = leave the env's primitives out
    // nullable (both or neither): n_envs + 1 offsets of each env's triangles
    // and edges when the primitives are ordered by env; oversize queries and
    // the oversize-entry lists are then searched within the query's env only
    const int* env_tri_start = nullptr;
    const int* env_edge_start = nullptr;
    // a contiguous range of the primitives: local point, edge and triangle i
    // are the global ones sv_base + i, edge_base + i, tri_base + i (every
    // other array above is indexed globally); output pairs hold global ids
    int sv_base = 0, edge_base = 0, tri_base = 0;
};

struct BroadPhase {
    // boxes
    DBuf<double> pbox, ebox, tbox;  // 6 per primitive: lo xyz, hi xyz
    DBuf<int> pcb, ecb, tcb;        // 6 per primitive: integer cell range lo xyz, hi xyz
    DBuf<uint32_t> tcnt, toff, ecnt, eoff;
    DBuf<uint64_t> key, key2;
    DBuf<uint32_t> val, val2;
    DBuf<uint64_t> ecell;  // sorted entry cell keys
    DBuf<int> eprim;       // sorted entry primitive ids
    DBuf<uint32_t> bstart, bend;
    DBuf<int> big_t, big_e, big_p, big_q;
    DBuf<uint32_t> pflag, pflagoff;
    DBuf<uint32_t> flag, flagoff;
    DBuf<uint32_t> qcnt_pt, qoff_pt, qcnt_ee, qoff_ee;
    DBuf<uint32_t> tmp;
    DBuf<int2> pt, ee;  // outputs: (sv, tri), (edge, edge)
    DBuf<int2> slot_pt, slot_ee;  // the counting pass's first hits per query
    DBuf<uint32_t> hcount;  // pinned-size mirror of counts on device
    uint32_t n_pt = 0, n_ee = 0;
    uint32_t* h_counts = nullptr;  // pinned host [4]

    // Runs the broad phase; n_pt / n_ee hold the counts afterwards (the call
    // synchronises the stream once to size the outputs).
    void run(Allocator* A, const BPView& v, cudaStream_t st);
    ~BroadPhase();
};

}  // namespace zema
