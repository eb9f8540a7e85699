// Device-side view of a scene.  All DOFs are 3-vector "nodes" stored AoS
// (x, y, z interleaved, 24 B per node):
//   soft vertex            -> 1 node (its position)
//   affine body (12 DOF)   -> 4 nodes (p', c1, c2, c3): p' the world position
//                             of the body's centre of mass, c_k = A e_k the
//                             columns of A.  A rest vertex x0' (relative to
//                             the centre of mass) maps to
//                             x = p' + x0'_0 c1 + x0'_1 c2 + x0'_2 c3,
//                             i.e. a weighted sum of 4 nodes with weights
//                             (1, x0'), and the affine mass matrix of Eq. 2
//                             becomes diag(m, S') (x) I3.
// Nodes, tets, affine bodies, surface vertices and edges are ordered by
// environment so that every per-environment quantity is a contiguous range.
#pragma once
#include "common.cuh"

namespace zema {

// A prismatic joint between two affine bodies (paper Sec. "Joint
// Constraints"): constants fixed at the scene's initial state.
struct JointDev {
    int n1, n2;          // first node of each body (p', then the columns of A)
    int fix1, fix2;      // body fixed (Dirichlet): its nodes take no gradient
    int env;
    double kappa;        // penalty stiffness
    double B1[9], B2[9]; // inverses of each body's initial A (row-major)
    double u1[3], u2[3]; // joint point minus the body's centre of mass, body rest frame
    double d1[3];        // unit axis in body 1's rest frame
};

struct Geo {
    int n_nodes, n_soft, n_aff, n_tets, n_sv, n_edges, n_tris, n_envs, n_units, n_bodies;
    double h, dhat, eps_v;
    // nodes
    const int* node_env;
    const uint8_t* node_fixed;
    const double* node_mass;        // lumped mass of soft nodes (0 for affine nodes)
    const int* env_node_start;      // n_envs + 1
    // tets (soft elasticity)
    const int4* tets;               // node indices
    const double* Dminv;            // 9 per tet, row-major inverse rest edge matrix
    const double* tvol;             // rest volume
    const double* tmu;              // Lame mu
    const double* tlam;             // Lame lambda
    const uint8_t* tmodel;          // material per tet: 0 Neo-Hookean, 1 St. Venant-Kirchhoff, 2 fixed corotated
    const double* spring_k;         // per node: spring stiffness (N/m, 0: none); null when no springs
    const double* spring_x;         // per node: spring target (3)
    const int* env_tet_start;
    // affine bodies
    const int* aff_node0;
    const int* aff_mode;            // 0 dynamic, 1 fixed, 2 kinematic
    const double* aff_m;
    const double* aff_S;            // 9: centred second moment integral rho x0' x0'^T
    const double* aff_vol;
    const double* aff_stiff;
    const double* aff_com;          // 3: centre of mass in the caller's rest frame
    const int* env_aff_start;
    // prismatic joints, ordered by env
    int n_joints;
    const JointDev* joints;
    const int* env_joint_start;
    const double* lamJ;             // 12 AL multipliers per joint
    // units of the block-Jacobi preconditioner: a soft node or an affine body
    const int* unit_kind;           // 0 soft node, 1 affine body
    const int* unit_idx;
    const int* env_unit_start;
    // surface
    const int* sv_node;             // soft: its node; affine: first node of the body
    const uint8_t* sv_aff;
    const double* sv_x0;            // 3 per sv: rest position relative to COM (affine)
    const double* sv_rest;          // 3 per sv: rest position (for the edge-edge mollifier threshold)
    const int* sv_body;
    const int* sv_env;
    const int* body_class;          // per body: 0 soft, 1 affine dynamic, 2 fixed, 3 kinematic
    const double* body_mu;          // friction coefficient per body
    const int2* edges;              // surface vertex ids
    const int3* tris;
    const double* edge_rest2;       // squared rest length per edge
    const int* env_sv_start;
    const int* env_edge_start;
    // soft node -> incident (tet * 4 + local) for the gradient gather
    const int* node_tet_ptr;
    const int* node_tet_idx;
    // static block-sparse pattern (3x3 blocks over nodes)
    const int* S_rowptr;
    const int* S_col;
    const int* S_src_ptr;           // per block: range into S_src
    const int* S_src;               // staging block index (tets first, then affine bodies)
    // nullable, per env: nonzero = the env's Newton solve has converged; the
    // per-iteration kernels then skip its elements, bodies, blocks, pairs and
    // energy terms (its results are not used until its next solve)
    const int* env_done = nullptr;
};

__device__ __forceinline__ bool env_is_done(const Geo& G, int env) { return G.env_done && G.env_done[env]; }

// world position of a surface vertex from node positions x
__device__ __forceinline__ V3 sv_pos(const Geo& G, const double* x, int s) {
    int n = G.sv_node[s];
    if (!G.sv_aff[s]) return ld3(x + 3 * (size_t)n);
    const double* w = G.sv_x0 + 3 * (size_t)s;
    V3 p = ld3(x + 3 * (size_t)n);
    V3 c1 = ld3(x + 3 * (size_t)(n + 1)), c2 = ld3(x + 3 * (size_t)(n + 2)), c3 = ld3(x + 3 * (size_t)(n + 3));
    return p + w[0] * c1 + w[1] * c2 + w[2] * c3;
}

// Number of nodes a surface vertex depends on, their ids and weights.
__device__ __forceinline__ int sv_nodes(const Geo& G, int s, int* nd, double* w) {
    int n = G.sv_node[s];
    if (!G.sv_aff[s]) {
        nd[0] = n;
        w[0] = 1.0;
        return 1;
    }
    const double* x0 = G.sv_x0 + 3 * (size_t)s;
    nd[0] = n;
    nd[1] = n + 1;
    nd[2] = n + 2;
    nd[3] = n + 3;
    w[0] = 1.0;
    w[1] = x0[0];
    w[2] = x0[1];
    w[3] = x0[2];
    return 4;
}

// A contact or friction pair record: 4 surface vertices and a kind.
struct PairRec {
    int s[4];
    int is_ee;
};

}  // namespace zema
