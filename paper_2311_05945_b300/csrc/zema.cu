// zema: C ABI and host orchestration of the soft-rigid coupled IPC time step.
//
// Per time step (paper section III): predictor (Eq. 1-3), lagged friction at
// x^t (Eq. 9-10), a CCD-filtered warm start, then projected Newton on
// B_t + D (Eq. 4, Eq. 11): spatial-hash broad phase, active pairs d < dhat,
// PSD-projected local Hessians (elastic, affine, barrier in the 12-dim pair
// space mapped by the coupling Jacobian of Eq. 6-8, friction), block-sparse
// assembly, block-Jacobi PCG, step-norm convergence test, swept broad phase +
// additive CCD bound, backtracking line search; then the velocity update
// (Eq. 11), kappa adaptation and the kinematic augmented-Lagrangian update
// (Eq. 13).  The host only sequences kernels and reads back counts, per-env
// energies and flags.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <numeric>
#include <tuple>
#include <vector>

#include "broadphase.cuh"
#include "kernels_misc.cuh"
#include "mlp.cuh"
#include "pcg_cluster.cuh"
#include "warmstart.cuh"

using namespace zema;

namespace {

struct TetIn {
    int env;
    std::vector<double> X, x0, v0;
    std::vector<int> T;
    double E, nu, rho, mu;
    int model = 0;                    // 0 Neo-Hookean, 1 St. Venant-Kirchhoff, 2 fixed corotated
    std::vector<int> spring_v;        // springs: body-local vertex, target (3 each), stiffness
    std::vector<double> spring_x;
    double spring_k = 0.0;
};
struct JointIn {
    int a1, a2;       // affine input indices
    double axis[3];   // unit axis in world coordinates at the initial state
    double kappa;     // <= 0: 1e3 x the mean of the two bodies' masses
};
struct AffIn {
    int env, mode;
    std::vector<double> V;
    std::vector<int> F;
    double q0[12], qd0[12];
    double rho, stiff, mu;
};

constexpr int TB = 256;

inline dim3 red_grid(int n_envs) { return dim3(kChunks, n_envs); }

}  // namespace

constexpr int kUpSlots = 128;  // pinned upload slots per scene (see zema_scene::h_up_i)

struct zema_scene {
    zema_scene_params P;
    Allocator A;
    cudaStream_t st = nullptr;
    std::string err;
    bool finalized = false;
    std::vector<TetIn> tin;
    std::vector<AffIn> ain;
    std::vector<std::pair<int, int>> bodies;  // body id -> (0 tet / 1 affine, index)

    // host copies needed at the boundary
    int n_envs = 1;
    std::vector<int> tet_body_node0;   // first node of each tet body
    std::vector<int> aff_node0_h;      // first node of each affine body
    std::vector<double> aff_com_h;     // 3 per affine body
    std::vector<int> aff_mode_h;
    std::vector<double> diag_h, tol_h; // per env
    std::vector<int> env_aff_start_h, env_node_start_h, env_sv_start_h, env_edge_start_h, env_tri_start_h;
    std::vector<double> node_mass_h, aff_m_in;  // host copies for the kappa rule
    int n_nodes = 0, n_soft = 0, n_aff = 0, n_tets = 0, n_sv = 0, n_edges = 0, n_tris = 0, n_units = 0;
    int n_sblocks = 0;
    double cell = 1.0;
    std::vector<int> kappa_ready;  // per env: kappa set (by rule or by user)
    bool first_step_done = false;

    // device geometry
    DBuf<int> node_env, env_node_start, env_tet_start, env_aff_start, env_unit_start, env_sv_start, env_edge_start;
    DBuf<int> env_tri_start;  // surface triangles are ordered by env too
    DBuf<uint8_t> tmodel;
    DBuf<double> spring_k, spring_x;  // per node (allocated with the first spring)
    bool has_springs = false;
    DBuf<uint8_t> node_fixed, sv_aff;
    DBuf<double> node_mass, Dminv, tvol, tmu, tlam, aff_m, aff_S, aff_vol, aff_stiff, aff_com, sv_x0, sv_rest,
        body_mu, edge_rest2;
    DBuf<int4> tets;
    DBuf<int> aff_node0, aff_mode, unit_kind, unit_idx, sv_node, sv_body, sv_env, body_class, node_tet_ptr,
        node_tet_idx, S_rowptr, S_col, S_src_ptr, S_src, S_diag;
    DBuf<int2> edges;
    DBuf<int3> tris;
    // state
    DBuf<double> x, v, xt, xhat, p, xtrial, g, b, r, z, pp, q, X, Xt, X1, stage_blk, stage_g, S_val, Minv_s, Minv_a;
    DBuf<double> pcg_work;  // work vectors of the grid-wide solve (6 x 3 n_nodes of the solve's type)
    DBuf<double> qtarget, lamA;
    std::vector<JointIn> jin;
    DBuf<JointDev> joints;
    DBuf<int> env_joint_start;
    DBuf<double> lamJ, lamJ_save;
    std::vector<int> joint_order;  // device joint -> input joint
    // per env
    DBuf<double> tol2_env;
    DBuf<double> kappa, kappa_min, alpha, E, dmin, part, part2, part3, part4, part5, part6, part7;
    DBuf<int> conv, pcg_iters, need, capflag, skip, pcg_refines, ls_skip;
    DBuf<int> tile_u0, tile_u1, tile_n0, tile_n1, tile_env, env_tile_start;
    DBuf<double> pt_a, pt_b, pt_c, pt_d, pt_e;
    int n_tiles = 0, pcg_grid = 0, pcg_grid_f = 0;
    // cluster PCG: CTAs per env (0 = not chosen yet, -1 = unavailable) and
    // its shared-memory layout bounds
    int pcgc_cs[2] = {0, 0};
    bool pcgc_tune[2] = {false, false};  // autotune the cluster size at the next solve
    bool pcgc_tuned_flag[2] = {false, false};  // the schedule came from the autotuner
    int pcgc_valid16[2] = {-1, -1};             // whether schedule 16 can run (-1: not checked yet)
    int n_sm = 0;
    std::vector<std::pair<int, float>> pcgc_tuned[2];  // (cluster size, solve ms) measured by the autotuner
    int pcgc_max_env_nodes = 0, pcgc_max_soft = 0, pcgc_max_aff = 0;
    std::vector<int> env_soft_h;  // soft nodes per env
    // size-binned schedules, per multiplier m: the envs of each cluster size
    // 1, 2, 4, 8, 16 (groups in that order) in one device list, and the 6
    // group offsets
    DBuf<int> pcgc_bin_list[5];
    std::vector<int> pcgc_bin_off[5];
    std::vector<int> S_rowptr_h;  // host copy of the static pattern's row pointers
    std::map<std::pair<int, int>, int> pcgc_cap;  // (value size, CTAs per env) -> staged slice capacity
    DBuf<double> tolv;
    // pair lists
    BroadPhase bp;
    DBuf<PairRec> cand, act, swept, lag, recs;
    DBuf<uint32_t> flag, flagoff, pt_env, ee_env, m_env, act_env, swept_env, lag_env, tmp32;
    DBuf<double> lag_w, lag_n, lag_c, pH, pG;
    DBuf<int> pflag;  // per active pair: its Hessian block awaits projection
    uint32_t n_act = 0, n_swept = 0, n_lag = 0;
    // contact assembly
    DBuf<uint32_t> cnt_blk, off_blk, cnt_g, off_g, bval, bval2, gval, gval2, head, hoff, seg;
    DBuf<uint64_t> bkey, bkey2, gkey, gkey2, ukey;
    DBuf<double> bstage, gstage, C_val, gsum;
    DBuf<int> C_rowptr, C_col;
    DBuf<float4> pk;  // the FP32 matrix packed for the cluster solve (k_pack_blocks)
    uint32_t n_cblocks = 0;
    bool n_cblocks_pending = false;  // the count waits in h32[8] for the next read-back
    DBuf<uint32_t> cnt_u;            // unique contact blocks and gradient nodes, on the device
    // pinned host scratch
    uint32_t* h32 = nullptr;
    double* hd = nullptr;
    int* hi = nullptr;
    double* h_alpha = nullptr;  // the line search's ACCD bounds, read back with its first trial
    // per-env host-to-device uploads go through a ring of pinned slots, so
    // that the host never rewrites a pinned buffer whose asynchronous copy
    // may not have run yet (a stream synchronises many times per ring turn)
    int* h_up_i = nullptr;
    double* h_up_d = nullptr;
    unsigned h_up_pos = 0;
    // a solve's iteration counts and status (pinned, 2 per env), read back
    // with the next round trip; its kernel name and value size for the
    // roofline's byte count
    int* h_pcg = nullptr;
    bool pcg_pending = false;
    // the cluster solve's launch order: envs by their last solve's cost
    // (iterations x nodes), largest first, so that the longest solves start
    // first and the launch does not end on one late long solve
    std::vector<double> env_cost;
    std::vector<int> env_order_h;
    DBuf<int> env_order;
    int pcg_pending_tsize = 0;
    bool pcg_pending_refines = false;  // the waiting read-back holds in-launch refinement counts
    const char* pcg_pending_kname = nullptr;
    Geo G{};
    // stats of the current call
    zema_step_stats S{};
    // host-side fault injection (zema_inject_fault): kind, the Newton
    // iteration of the call it fires at, the call's Newton iteration count,
    // the kind armed for the current iteration, and the device flag / status
    // word the injection kernels read and write
    int fault_kind = 0, fault_at = 0, newton_count = 0, fault_armed = 0;
    DBuf<int> fault_dev;
    // per-step scratch
    DBuf<double> dirw, lam_save;
    // kinematic multipliers at the end of the step before the last one (the
    // extrapolation's second point), and the step-start copies of lambda_A
    // and of it, put back by a full restore_step
    DBuf<double> lamA_prev, lam_hist;
    std::vector<double> dmin_last;
    // the step-start values of what a step may change before it completes
    // (kappa, kappa_min and their flags, d_min), put back by restore_step
    DBuf<double> kap_save;
    std::vector<int> kappa_ready_save;
    std::vector<double> dmin_last_save;
    bool first_step_done_save = false;
    // learned warm start: network, soft-vertex list (node order) with their
    // tet body, per-body node range / rest half-diagonal / centroid, features
    Mlp* ws_net = nullptr;
    Mlp* ws_anet = nullptr;  // per dynamic affine body (40 -> 12)
    int ws_ns = 0, ws_nb = 0, ws_na = 0;
    DBuf<int> ws_aff;                       // dynamic affine bodies (device index)
    DBuf<double> ws_aR, ws_envc, ws_envd;   // their rest half-diagonals; env bbox centres and diagonals
    DBuf<float> ws_afeat, ws_aout;
    DBuf<int> body_env;      // env of every body (caller ids), for force sensing
    DBuf<double> body_force;
    float* rec_afeat = nullptr;  // caller's device buffers while recording the affine rows
    float* rec_atarg = nullptr;
    DBuf<int> ws_soft, ws_body, tb_node0, tb_nv;
    DBuf<double> tb_R, tb_c;
    DBuf<unsigned long long> ws_best;
    DBuf<float> ws_feat, ws_out;
    float* rec_feat = nullptr;  // caller's device buffers while recording
    float* rec_targ = nullptr;
    mutable std::vector<int> aff_dev_of_input;  // device index of each affine body (order of addition)
    // size-binned solves: one stream per cluster size, the fork event and
    // the join events
    cudaStream_t bin_st[5] = {};
    cudaEvent_t bin_fork = nullptr, bin_join[5] = {};
    // zema_set_kinematic_targets: pinned staging of (device affine index,
    // 12 target values) records, their device copy, and the event after the
    // copy out of the staging (waited on before the staging is rewritten)
    // zema_get/set_scene_state: per body (order of addition) its first node,
    // vertex count (tet bodies; -1 for affine bodies), offset in the flat
    // state, fixed flag and (affine) centre of mass; and the device copy of
    // the flat state
    DBuf<int> sst_node0, sst_nv, sst_fixed;
    DBuf<int64_t> sst_off;
    DBuf<double> sst_com, sst_buf;
    int64_t sst_n = -1;
    double* h_kin = nullptr;
    size_t h_kin_cap = 0;
    DBuf<double> kin_up;
    cudaEvent_t kin_ev = nullptr;

    ~zema_scene() {
        if (h_kin) cudaFreeHost(h_kin);
        for (int k = 0; k < 5; ++k) {
            if (bin_st[k]) cudaStreamDestroy(bin_st[k]);
            if (bin_join[k]) cudaEventDestroy(bin_join[k]);
        }
        if (bin_fork) cudaEventDestroy(bin_fork);
        if (kin_ev) cudaEventDestroy(kin_ev);
        delete ws_net;
        delete ws_anet;
        if (h32) cudaFreeHost(h32);
        if (hd) cudaFreeHost(hd);
        if (hi) cudaFreeHost(hi);
        if (h_alpha) cudaFreeHost(h_alpha);
        if (h_up_i) cudaFreeHost(h_up_i);
        if (h_up_d) cudaFreeHost(h_up_d);
        if (h_pcg) cudaFreeHost(h_pcg);
    }
};

namespace {

void fail(int status, const std::string& m) { throw ZemaError{status, m}; }

// n_envs values into device memory through the next pinned ring slot (see
// zema_scene::h_up_i)
void upload_env_ints(zema_scene* s, int* dst, const int* src) {
    const int NE = s->n_envs;
    int* slot = s->h_up_i + (size_t)(s->h_up_pos++ % kUpSlots) * NE;
    std::memcpy(slot, src, NE * sizeof(int));
    ZCHECK(cudaMemcpyAsync(dst, slot, NE * sizeof(int), cudaMemcpyHostToDevice, s->st));
}
void upload_env_doubles(zema_scene* s, double* dst, const double* src) {
    const int NE = s->n_envs;
    double* slot = s->h_up_d + (size_t)(s->h_up_pos++ % kUpSlots) * NE;
    std::memcpy(slot, src, NE * sizeof(double));
    ZCHECK(cudaMemcpyAsync(dst, slot, NE * sizeof(double), cudaMemcpyHostToDevice, s->st));
}

template <class T>
void up(zema_scene* s, DBuf<T>& d, const std::vector<T>& h) {
    d.upload(&s->A, h);
}

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------
// Host-side fault injection (zema_inject_fault).  The host arms a device flag
// for one Newton iteration; these kernels read it and report a failure
// through the same status words the real failures use.  Nothing is made to
// fault, trap or hang.
// ---------------------------------------------------------------------------
// the status word flag[1] of an armed flag[0]: ZEMA_ERR_FAULT_INJECTED
__global__ void k_fault_status_word(int* flag) {
    if (threadIdx.x == 0 && flag[0]) flag[1] = ZEMA_ERR_FAULT_INJECTED;
}
// an armed flag marks every env's linear solve as having met a non-finite
// value (the solve kernels' own conv code 2)
__global__ void k_fault_solve_status(const int* flag, int* conv, int n_envs) {
    if (!flag[0]) return;
    for (int e = threadIdx.x; e < n_envs; e += blockDim.x) conv[e] = 2;
}

// ---------------------------------------------------------------------------
// Scene precompute kernels (rest shapes, masses)
// ---------------------------------------------------------------------------
__global__ void k_tet_rest(const double* Xr, const int4* tets, int nt, double* Dminv, double* vol, int* bad) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int4 T = tets[t];
    const double* a = Xr + 3 * (size_t)T.x;
    double Dm[9];
    const double* o[3] = {Xr + 3 * (size_t)T.y, Xr + 3 * (size_t)T.z, Xr + 3 * (size_t)T.w};
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 3; ++r) Dm[3 * r + c] = o[c][r] - a[r];
    double det;
    inv3(Dm, Dminv + 9 * (size_t)t);
    det = Dm[0] * (Dm[4] * Dm[8] - Dm[5] * Dm[7]) - Dm[1] * (Dm[3] * Dm[8] - Dm[5] * Dm[6]) +
          Dm[2] * (Dm[3] * Dm[7] - Dm[4] * Dm[6]);
    vol[t] = det / 6.0;
    if (!(det > 0.0)) atomicMax(bad, 1);
}

// lumped vertex mass: sum over incident tets of rho V / 4
__global__ void k_lumped_mass(const int* ptr, const int* idx, const double* vol, const double* trho, int n,
                              double* mass) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    double m = 0.0;
    for (int k = ptr[v]; k < ptr[v + 1]; ++k) {
        int t = idx[k] >> 2;
        m += trho[t] * vol[t] * 0.25;
    }
    mass[v] = m;
}

// Mass properties of an affine body from its closed surface (Eq. 2):
// integrals of 1, x0, x0 x0^T over the enclosed volume via the tetrahedra
// (origin, a, b, c) of each outward triangle.  One block per body.
__global__ void k_affine_mass(const double* V, const int* F, const int* f_ptr, const int* v_off, const double* rho,
                              int nb, double* out /* 13 per body: vol, m1(3), m2(9) */) {
    int b = blockIdx.x;
    if (b >= nb) return;
    __shared__ double sh[32];
    double acc[13];
    for (int i = 0; i < 13; ++i) acc[i] = 0.0;
    const double* Vb = V + 3 * (size_t)v_off[b];
    for (int f = f_ptr[b] + threadIdx.x; f < f_ptr[b + 1]; f += blockDim.x) {
        const double* a = Vb + 3 * (size_t)F[3 * f];
        const double* c1 = Vb + 3 * (size_t)F[3 * f + 1];
        const double* c2 = Vb + 3 * (size_t)F[3 * f + 2];
        double vol = (a[0] * (c1[1] * c2[2] - c1[2] * c2[1]) - a[1] * (c1[0] * c2[2] - c1[2] * c2[0]) +
                      a[2] * (c1[0] * c2[1] - c1[1] * c2[0])) / 6.0;
        double s[3];
        for (int i = 0; i < 3; ++i) s[i] = a[i] + c1[i] + c2[i];
        acc[0] += vol;
        for (int i = 0; i < 3; ++i) acc[1 + i] += vol * s[i] * 0.25;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                acc[4 + 3 * i + j] += vol / 20.0 * (a[i] * a[j] + c1[i] * c1[j] + c2[i] * c2[j] + s[i] * s[j]);
    }
    for (int i = 0; i < 13; ++i) {
        double t = block_sum<kRedThreads>(acc[i], sh);
        if (threadIdx.x == 0) out[13 * (size_t)b + i] = t * (i == 0 ? 1.0 : rho[b]);
    }
}

// ---------------------------------------------------------------------------
// finalize: layout, topology, static pattern, uploads
// ---------------------------------------------------------------------------
// device spring arrays of a tet body from its TetIn (zero stiffness elsewhere)
void upload_springs(zema_scene* s, int tb) {
    const TetIn& B = s->tin[tb];
    const size_t nN = (size_t)s->n_nodes;
    if (!s->has_springs) {
        s->spring_k.ensure(&s->A, nN + 1);
        s->spring_x.ensure(&s->A, 3 * nN + 3);
        ZCHECK(cudaMemsetAsync(s->spring_k.p, 0, (nN + 1) * sizeof(double), s->st));
        ZCHECK(cudaMemsetAsync(s->spring_x.p, 0, (3 * nN + 3) * sizeof(double), s->st));
        s->has_springs = true;
        s->G.spring_k = s->spring_k.p;
        s->G.spring_x = s->spring_x.p;
    }
    const int n0 = s->tet_body_node0[tb], nv = (int)(B.X.size() / 3);
    std::vector<double> k(nv, 0.0), x(3 * (size_t)nv, 0.0);
    for (size_t i = 0; i < B.spring_v.size(); ++i) {
        const int v = B.spring_v[i];
        k[v] = B.spring_k;
        for (int j = 0; j < 3; ++j) x[3 * (size_t)v + j] = B.spring_x[3 * i + j];
    }
    ZCHECK(cudaMemcpyAsync(s->spring_k.p + n0, k.data(), nv * sizeof(double), cudaMemcpyHostToDevice, s->st));
    ZCHECK(cudaMemcpyAsync(s->spring_x.p + 3 * (size_t)n0, x.data(), 3 * (size_t)nv * sizeof(double),
                           cudaMemcpyHostToDevice, s->st));
    ZCHECK(cudaStreamSynchronize(s->st));
}

void build(zema_scene* s) {
    cudaStream_t st = s->st;
    Allocator* A = &s->A;
    const int NE = s->n_envs;
    if (s->bodies.empty()) fail(ZEMA_ERR_INVALID_ARG, "scene has no bodies");
    // ---- node layout by env: soft bodies then affine bodies
    std::vector<int> tet_order, aff_order;
    for (int e = 0; e < NE; ++e)
        for (size_t i = 0; i < s->tin.size(); ++i)
            if (s->tin[i].env == e) tet_order.push_back((int)i);
    for (int e = 0; e < NE; ++e)
        for (size_t i = 0; i < s->ain.size(); ++i)
            if (s->ain[i].env == e) aff_order.push_back((int)i);
    s->tet_body_node0.assign(s->tin.size(), 0);
    s->aff_node0_h.assign(s->ain.size(), 0);
    std::vector<int> node_env_h, env_node_start(NE + 1, 0), env_tet_start(NE + 1, 0), env_aff_start(NE + 1, 0);
    std::vector<uint8_t> node_fixed_h;
    std::vector<int4> tets_h;
    std::vector<double> trho_h, tmu_h, tlam_h, xrest_h, x_h, v_h;
    std::vector<uint8_t> tmodel_h;
    std::vector<int> aff_perm;  // affine device index -> input index
    {
        size_t ti = 0, ai = 0;
        for (int e = 0; e < NE; ++e) {
            env_node_start[e] = (int)node_env_h.size();
            env_tet_start[e] = (int)tets_h.size();
            for (; ti < tet_order.size() && s->tin[tet_order[ti]].env == e; ++ti) {
                TetIn& B = s->tin[tet_order[ti]];
                int n0 = (int)node_env_h.size();
                s->tet_body_node0[tet_order[ti]] = n0;
                size_t nv = B.X.size() / 3;
                for (size_t k = 0; k < nv; ++k) {
                    node_env_h.push_back(e);
                    node_fixed_h.push_back(0);
                    for (int j = 0; j < 3; ++j) {
                        xrest_h.push_back(B.X[3 * k + j]);
                        x_h.push_back(B.x0[3 * k + j]);
                        v_h.push_back(B.v0[3 * k + j]);
                    }
                }
                double mu = B.E / (2.0 * (1.0 + B.nu)), lam = B.E * B.nu / ((1.0 + B.nu) * (1.0 - 2.0 * B.nu));
                for (size_t t = 0; t < B.T.size() / 4; ++t) {
                    tets_h.push_back(make_int4(n0 + B.T[4 * t], n0 + B.T[4 * t + 1], n0 + B.T[4 * t + 2],
                                               n0 + B.T[4 * t + 3]));
                    trho_h.push_back(B.rho);
                    tmu_h.push_back(mu);
                    tlam_h.push_back(lam);
                    tmodel_h.push_back((uint8_t)B.model);
                }
            }
            env_aff_start[e] = (int)aff_perm.size();
            for (; ai < aff_order.size() && s->ain[aff_order[ai]].env == e; ++ai) {
                int n0 = (int)node_env_h.size();
                s->aff_node0_h[aff_order[ai]] = n0;
                aff_perm.push_back(aff_order[ai]);
                for (int k = 0; k < 4; ++k) {
                    node_env_h.push_back(e);
                    node_fixed_h.push_back(s->ain[aff_order[ai]].mode == 1 ? 1 : 0);
                    for (int j = 0; j < 3; ++j) {
                        xrest_h.push_back(0.0);
                        x_h.push_back(0.0);
                        v_h.push_back(0.0);
                    }
                }
            }
        }
        env_node_start[NE] = (int)node_env_h.size();
        env_tet_start[NE] = (int)tets_h.size();
        env_aff_start[NE] = (int)aff_perm.size();
    }
    s->n_nodes = (int)node_env_h.size();
    s->n_tets = (int)tets_h.size();
    s->n_aff = (int)aff_perm.size();
    s->env_node_start_h = env_node_start;
    s->env_aff_start_h = env_aff_start;
    int nN = s->n_nodes;
    // soft node count (nodes before the affine ones within each env are soft)
    std::vector<double> node_mass_h(nN, 0.0);
    // ---- node -> incident tets (sorted by tet, local)
    std::vector<int> ntp(nN + 1, 0), nti;
    for (int t = 0; t < s->n_tets; ++t) {
        int4 T = tets_h[t];
        ntp[T.x + 1]++;
        ntp[T.y + 1]++;
        ntp[T.z + 1]++;
        ntp[T.w + 1]++;
    }
    for (int i = 0; i < nN; ++i) ntp[i + 1] += ntp[i];
    nti.assign(ntp[nN], 0);
    {
        std::vector<int> cur(ntp.begin(), ntp.end() - 1);
        for (int t = 0; t < s->n_tets; ++t) {
            int4 T = tets_h[t];
            int ids[4] = {T.x, T.y, T.z, T.w};
            for (int k = 0; k < 4; ++k) nti[cur[ids[k]]++] = 4 * t + k;
        }
    }
    // ---- surface: soft boundary faces, affine meshes
    std::vector<int> sv_node_h, sv_body_h, sv_env_h;
    std::vector<uint8_t> sv_aff_h;
    std::vector<double> sv_rest_h, sv_x0_h;
    std::vector<int2> edges_h;
    std::vector<int3> tris_h;
    std::vector<int> env_sv_start(NE + 1, 0), env_edge_start(NE + 1, 0), env_tri_start(NE + 1, 0);
    std::vector<int> body_id_of_tet(s->tin.size()), body_id_of_aff(s->ain.size());
    for (size_t b = 0; b < s->bodies.size(); ++b) {
        if (s->bodies[b].first == 0)
            body_id_of_tet[s->bodies[b].second] = (int)b;
        else
            body_id_of_aff[s->bodies[b].second] = (int)b;
    }
    // affine mass properties are needed for sv_x0: computed on the device
    // below; the rest-frame positions are filled after that.
    std::vector<int> sv_aff_body;  // device affine index per sv (or -1)
    std::vector<std::vector<int3>> env_tris(NE);
    {
        size_t ti = 0, ai = 0;
        static const int FL[4][3] = {{0, 2, 1}, {0, 1, 3}, {0, 3, 2}, {1, 2, 3}};
        for (int e = 0; e < NE; ++e) {
            env_sv_start[e] = (int)sv_node_h.size();
            std::vector<int3> etris;
            for (; ti < tet_order.size() && s->tin[tet_order[ti]].env == e; ++ti) {
                TetIn& B = s->tin[tet_order[ti]];
                int n0 = s->tet_body_node0[tet_order[ti]];
                std::map<std::tuple<int, int, int>, std::pair<int, std::tuple<int, int, int>>> faces;
                for (size_t t = 0; t < B.T.size() / 4; ++t) {
                    const int* T = &B.T[4 * t];
                    for (int f = 0; f < 4; ++f) {
                        int a = T[FL[f][0]], c = T[FL[f][1]], d = T[FL[f][2]];
                        int k[3] = {a, c, d};
                        std::sort(k, k + 3);
                        auto key = std::make_tuple(k[0], k[1], k[2]);
                        auto it = faces.find(key);
                        if (it == faces.end())
                            faces[key] = {1, std::make_tuple(a, c, d)};
                        else
                            it->second.first++;
                    }
                }
                std::map<int, int> local_sv;
                std::vector<std::tuple<int, int, int>> ft;
                for (auto& kv : faces)
                    if (kv.second.first == 1) ft.push_back(kv.second.second);
                for (auto& f : ft) {
                    local_sv[std::get<0>(f)] = 0;
                    local_sv[std::get<1>(f)] = 0;
                    local_sv[std::get<2>(f)] = 0;
                }
                for (auto& kv : local_sv) {
                    kv.second = (int)sv_node_h.size();
                    sv_node_h.push_back(n0 + kv.first);
                    sv_aff_h.push_back(0);
                    sv_body_h.push_back(body_id_of_tet[tet_order[ti]]);
                    sv_env_h.push_back(e);
                    sv_aff_body.push_back(-1);
                    for (int j = 0; j < 3; ++j) sv_rest_h.push_back(B.X[3 * kv.first + j]);
                }
                for (auto& f : ft)
                    etris.push_back(make_int3(local_sv[std::get<0>(f)], local_sv[std::get<1>(f)], local_sv[std::get<2>(f)]));
            }
            for (; ai < aff_order.size() && s->ain[aff_order[ai]].env == e; ++ai) {
                AffIn& B = s->ain[aff_order[ai]];
                int sv0 = (int)sv_node_h.size();
                int dev_idx = (int)ai;
                for (size_t k = 0; k < B.V.size() / 3; ++k) {
                    sv_node_h.push_back(s->aff_node0_h[aff_order[ai]]);
                    sv_aff_h.push_back(1);
                    sv_body_h.push_back(body_id_of_aff[aff_order[ai]]);
                    sv_env_h.push_back(e);
                    sv_aff_body.push_back(dev_idx);
                    for (int j = 0; j < 3; ++j) sv_rest_h.push_back(B.V[3 * k + j]);
                }
                for (size_t f = 0; f < B.F.size() / 3; ++f)
                    etris.push_back(make_int3(sv0 + B.F[3 * f], sv0 + B.F[3 * f + 1], sv0 + B.F[3 * f + 2]));
            }
            // edges of this env, unique, ordered by (min, max)
            env_edge_start[e] = (int)edges_h.size();
            std::vector<std::pair<int, int>> ed;
            for (auto& t : etris) {
                int v3_[3] = {t.x, t.y, t.z};
                for (int k = 0; k < 3; ++k) {
                    int a = v3_[k], c = v3_[(k + 1) % 3];
                    ed.push_back({std::min(a, c), std::max(a, c)});
                }
            }
            std::sort(ed.begin(), ed.end());
            ed.erase(std::unique(ed.begin(), ed.end()), ed.end());
            for (auto& pr : ed) edges_h.push_back(make_int2(pr.first, pr.second));
            env_tri_start[e] = (int)tris_h.size();
            for (auto& t : etris) tris_h.push_back(t);
        }
        env_sv_start[NE] = (int)sv_node_h.size();
        env_edge_start[NE] = (int)edges_h.size();
        env_tri_start[NE] = (int)tris_h.size();
    }
    s->n_sv = (int)sv_node_h.size();
    s->n_edges = (int)edges_h.size();
    s->n_tris = (int)tris_h.size();
    s->env_sv_start_h = env_sv_start;
    s->env_edge_start_h = env_edge_start;
    s->env_tri_start_h = env_tri_start;
    std::vector<double> edge_rest2_h(s->n_edges);
    double sum_len = 0.0;
    for (int i = 0; i < s->n_edges; ++i) {
        double d2 = 0.0;
        for (int j = 0; j < 3; ++j) {
            double d = sv_rest_h[3 * edges_h[i].x + j] - sv_rest_h[3 * edges_h[i].y + j];
            d2 += d * d;
        }
        edge_rest2_h[i] = d2;
        sum_len += std::sqrt(d2);
    }
    double mean_len = s->n_edges ? sum_len / s->n_edges : s->P.dhat;
    s->cell = s->P.cell_size > 0.0 ? s->P.cell_size : std::max(mean_len, s->P.dhat);
    // ---- bodies
    std::vector<int> body_class_h(s->bodies.size());
    std::vector<double> body_mu_h(s->bodies.size());
    for (size_t b = 0; b < s->bodies.size(); ++b) {
        auto k = s->bodies[b];
        if (k.first == 0) {
            body_class_h[b] = 0;
            body_mu_h[b] = s->tin[k.second].mu;
        } else {
            int m = s->ain[k.second].mode;
            body_class_h[b] = m == 0 ? 1 : (m == 1 ? 2 : 3);
            body_mu_h[b] = s->ain[k.second].mu;
        }
    }
    // ---- units: per env soft nodes then affine bodies
    std::vector<int> unit_kind_h, unit_idx_h, env_unit_start(NE + 1, 0);
    for (int e = 0; e < NE; ++e) {
        env_unit_start[e] = (int)unit_kind_h.size();
        for (int n = env_node_start[e]; n < env_node_start[e + 1]; ++n) {
            bool is_aff = false;
            for (int a = env_aff_start[e]; a < env_aff_start[e + 1]; ++a) {
                int n0 = s->aff_node0_h[aff_perm[a]];
                if (n >= n0 && n < n0 + 4) is_aff = true;
            }
            if (!is_aff) {
                unit_kind_h.push_back(0);
                unit_idx_h.push_back(n);
            }
        }
        for (int a = env_aff_start[e]; a < env_aff_start[e + 1]; ++a) {
            unit_kind_h.push_back(1);
            unit_idx_h.push_back(a);
        }
    }
    env_unit_start[NE] = (int)unit_kind_h.size();
    s->n_units = (int)unit_kind_h.size();
    // PCG tiles of the grid-wide solve: one tile per affine unit, and runs of
    // <= kTileUnits consecutive soft units of one env with their node range,
    // sized so that all tiles together fill the resident blocks of the
    // cooperative launch once (every SM gets the same number of blocks; 16 to
    // 256 units, so a block's threads each own about one unit)
    int kTileUnits = 16;
    {
        int dev = 0, nsm = 148, per_f = 4, per_d = 4;
        if (cudaGetDevice(&dev) == cudaSuccess) {
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_f, k_pcg_persistent<float>, 256, 4096);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_d, k_pcg_persistent<double>, 256, 4096);
        }
        cudaGetLastError();
        size_t n_soft_units = 0;
        for (int k : unit_kind_h) n_soft_units += k == 0;
        const long long slots = (long long)std::max(1, std::min(per_f, per_d)) * nsm - (long long)s->n_aff;
        const size_t soft_tiles = (size_t)std::max(1LL, slots);
        const int want = (int)((n_soft_units + soft_tiles - 1) / soft_tiles);
        kTileUnits = std::max(16, std::min(256, want));
    }
    std::vector<int> tu0, tu1, tn0, tn1, tenv, etile(NE + 1, 0);
    for (int e = 0; e < NE; ++e) {
        etile[e] = (int)tu0.size();
        // runs of <= kTileUnits soft units; every affine unit a tile of its own
        for (int u = env_unit_start[e], ue; u < env_unit_start[e + 1]; u = ue) {
            ue = u + 1;
            if (unit_kind_h[u] == 0)
                while (ue < env_unit_start[e + 1] && ue - u < kTileUnits && unit_kind_h[ue] == 0) ++ue;
            auto first_node = [&](int uu) {
                return unit_kind_h[uu] == 0 ? unit_idx_h[uu] : s->aff_node0_h[aff_perm[unit_idx_h[uu]]];
            };
            auto last_node = [&](int uu) { return first_node(uu) + (unit_kind_h[uu] == 0 ? 1 : 4); };
            tu0.push_back(u);
            tu1.push_back(ue);
            tn0.push_back(first_node(u));
            tn1.push_back(last_node(ue - 1));
            tenv.push_back(e);
        }
    }
    etile[NE] = (int)tu0.size();
    s->n_tiles = (int)tu0.size();
    for (int e = 0; e < NE; ++e) {
        int na = env_aff_start[e + 1] - env_aff_start[e];
        int nsoft = (env_node_start[e + 1] - env_node_start[e]) - 4 * na;
        s->pcgc_max_env_nodes = std::max(s->pcgc_max_env_nodes, env_node_start[e + 1] - env_node_start[e]);
        s->pcgc_max_soft = std::max(s->pcgc_max_soft, nsoft);
        s->pcgc_max_aff = std::max(s->pcgc_max_aff, na);
        s->env_soft_h.push_back(nsoft);
    }
    up(s, s->tile_u0, tu0);
    up(s, s->tile_u1, tu1);
    up(s, s->tile_n0, tn0);
    up(s, s->tile_n1, tn1);
    up(s, s->tile_env, tenv);
    up(s, s->env_tile_start, etile);
    for (DBuf<double>* b : {&s->pt_a, &s->pt_b, &s->pt_c, &s->pt_d, &s->pt_e}) b->ensure(A, s->n_tiles + 1);
    // ---- static pattern
    std::vector<std::vector<int>> rows(nN);
    for (int n = 0; n < nN; ++n) rows[n].push_back(n);
    for (auto& T : tets_h) {
        int ids[4] = {T.x, T.y, T.z, T.w};
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) rows[ids[i]].push_back(ids[j]);
    }
    std::vector<int> aff_node0_dev(s->n_aff), aff_mode_dev(s->n_aff);
    for (int a = 0; a < s->n_aff; ++a) {
        aff_node0_dev[a] = s->aff_node0_h[aff_perm[a]];
        aff_mode_dev[a] = s->ain[aff_perm[a]].mode;
        if (aff_mode_dev[a] == 1) continue;
        int n0 = aff_node0_dev[a];
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) rows[n0 + i].push_back(n0 + j);
    }
    // prismatic joints: ordered by env; every pair of free nodes of the two
    // bodies couples (8 x 8 blocks per joint)
    s->joint_order.clear();
    for (int e = 0; e < NE; ++e)
        for (size_t j = 0; j < s->jin.size(); ++j)
            if (s->ain[s->jin[j].a1].env == e) s->joint_order.push_back((int)j);
    auto joint_nodes = [&](int jd, int* nodes) {
        const JointIn& J = s->jin[s->joint_order[jd]];
        const int n1 = s->aff_node0_h[J.a1], n2 = s->aff_node0_h[J.a2];
        for (int k = 0; k < 4; ++k) {
            nodes[k] = s->ain[J.a1].mode == 1 ? -1 : n1 + k;
            nodes[4 + k] = s->ain[J.a2].mode == 1 ? -1 : n2 + k;
        }
    };
    for (int jd = 0; jd < (int)s->joint_order.size(); ++jd) {
        int nodes[8];
        joint_nodes(jd, nodes);
        for (int i = 0; i < 8; ++i)
            for (int j = 0; j < 8; ++j)
                if (nodes[i] >= 0 && nodes[j] >= 0) rows[nodes[i]].push_back(nodes[j]);
    }
    std::vector<int> S_rowptr_h(nN + 1, 0), S_col_h, S_diag_h(nN);
    for (int n = 0; n < nN; ++n) {
        std::sort(rows[n].begin(), rows[n].end());
        rows[n].erase(std::unique(rows[n].begin(), rows[n].end()), rows[n].end());
        S_rowptr_h[n + 1] = S_rowptr_h[n] + (int)rows[n].size();
        for (int c : rows[n]) S_col_h.push_back(c);
    }
    auto blk = [&](int r, int c) {
        auto it = std::lower_bound(S_col_h.begin() + S_rowptr_h[r], S_col_h.begin() + S_rowptr_h[r + 1], c);
        return (int)(it - S_col_h.begin());
    };
    for (int n = 0; n < nN; ++n) S_diag_h[n] = blk(n, n);
    s->n_sblocks = (int)S_col_h.size();
    std::vector<std::vector<int>> src(s->n_sblocks);
    for (int t = 0; t < s->n_tets; ++t) {
        int4 T = tets_h[t];
        int ids[4] = {T.x, T.y, T.z, T.w};
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) src[blk(ids[i], ids[j])].push_back(16 * t + 4 * i + j);
    }
    for (int a = 0; a < s->n_aff; ++a) {
        if (aff_mode_dev[a] == 1) continue;
        int n0 = aff_node0_dev[a];
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) src[blk(n0 + i, n0 + j)].push_back(16 * s->n_tets + 16 * a + 4 * i + j);
    }
    for (int jd = 0; jd < (int)s->joint_order.size(); ++jd) {
        int nodes[8];
        joint_nodes(jd, nodes);
        for (int i = 0; i < 8; ++i)
            for (int j = 0; j < 8; ++j)
                if (nodes[i] >= 0 && nodes[j] >= 0)
                    src[blk(nodes[i], nodes[j])].push_back(16 * (s->n_tets + s->n_aff) + 64 * jd + 8 * i + j);
    }
    std::vector<int> S_src_ptr_h(s->n_sblocks + 1, 0), S_src_h;
    for (int k = 0; k < s->n_sblocks; ++k) {
        std::sort(src[k].begin(), src[k].end());
        S_src_ptr_h[k + 1] = S_src_ptr_h[k] + (int)src[k].size();
        for (int q : src[k]) S_src_h.push_back(q);
    }
    // ---- uploads
    up(s, s->node_env, node_env_h);
    up(s, s->node_fixed, node_fixed_h);
    up(s, s->env_node_start, env_node_start);
    up(s, s->env_tet_start, env_tet_start);
    up(s, s->env_aff_start, env_aff_start);
    up(s, s->env_unit_start, env_unit_start);
    up(s, s->env_sv_start, env_sv_start);
    up(s, s->env_edge_start, env_edge_start);
    up(s, s->env_tri_start, env_tri_start);
    up(s, s->tets, tets_h);
    up(s, s->tmu, tmu_h);
    up(s, s->tlam, tlam_h);
    up(s, s->tmodel, tmodel_h);
    up(s, s->aff_node0, aff_node0_dev);
    up(s, s->aff_mode, aff_mode_dev);
    up(s, s->unit_kind, unit_kind_h);
    up(s, s->unit_idx, unit_idx_h);
    up(s, s->sv_node, sv_node_h);
    up(s, s->sv_aff, sv_aff_h);
    up(s, s->sv_body, sv_body_h);
    up(s, s->sv_env, sv_env_h);
    up(s, s->sv_rest, sv_rest_h);
    up(s, s->body_class, body_class_h);
    up(s, s->body_mu, body_mu_h);
    up(s, s->edges, edges_h);
    up(s, s->tris, tris_h);
    up(s, s->edge_rest2, edge_rest2_h);
    up(s, s->node_tet_ptr, ntp);
    up(s, s->node_tet_idx, nti);
    up(s, s->S_rowptr, S_rowptr_h);
    s->S_rowptr_h = S_rowptr_h;
    up(s, s->S_col, S_col_h);
    up(s, s->S_src_ptr, S_src_ptr_h);
    up(s, s->S_src, S_src_h);
    up(s, s->S_diag, S_diag_h);
    // ---- rest-shape precompute on the device
    DBuf<double> xrest_d, trho_d;
    up(s, xrest_d, xrest_h);
    up(s, trho_d, trho_h);
    s->Dminv.ensure(A, 9 * (size_t)s->n_tets + 9);
    s->tvol.ensure(A, s->n_tets + 1);
    s->node_mass.ensure(A, nN + 1);
    DBuf<int> bad;
    bad.ensure(A, 1);
    ZCHECK(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    if (s->n_tets) ZL(k_tet_rest, div_up(s->n_tets, TB), TB, 0, st)(xrest_d.p, s->tets.p, s->n_tets, s->Dminv.p, s->tvol.p, bad.p);
    ZLAUNCH();
    ZL(k_lumped_mass, div_up(nN, TB), TB, 0, st)(s->node_tet_ptr.p, s->node_tet_idx.p, s->tvol.p, trho_d.p, nN, s->node_mass.p);
    ZLAUNCH();
    // affine mass properties
    std::vector<double> Vall;
    std::vector<int> Fall, fptr(s->n_aff + 1, 0), voff(s->n_aff, 0);
    std::vector<double> arho(s->n_aff);
    for (int a = 0; a < s->n_aff; ++a) {
        AffIn& B = s->ain[aff_perm[a]];
        voff[a] = (int)(Vall.size() / 3);
        Vall.insert(Vall.end(), B.V.begin(), B.V.end());
        Fall.insert(Fall.end(), B.F.begin(), B.F.end());
        fptr[a + 1] = (int)(Fall.size() / 3);
        arho[a] = B.rho;
    }
    std::vector<double> mp(13 * (size_t)s->n_aff + 13, 0.0);
    if (s->n_aff) {
        DBuf<double> Vd, rhod, mpd;
        DBuf<int> Fd, fpd, vod;
        up(s, Vd, Vall);
        up(s, Fd, Fall);
        up(s, fpd, fptr);
        up(s, vod, voff);
        up(s, rhod, arho);
        mpd.ensure(A, mp.size());
        ZL(k_affine_mass, s->n_aff, kRedThreads, 0, st)(Vd.p, Fd.p, fpd.p, vod.p, rhod.p, s->n_aff, mpd.p);
        ZLAUNCH();
        ZCHECK(cudaMemcpyAsync(mp.data(), mpd.p, mp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    int bad_h = 0;
    ZCHECK(cudaMemcpyAsync(&bad_h, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaStreamSynchronize(st));
    if (bad_h) fail(ZEMA_ERR_INVERTED_INPUT, "a rest tetrahedron has non-positive volume");
    s->node_mass_h.assign(nN, 0.0);
    ZCHECK(cudaMemcpy(s->node_mass_h.data(), s->node_mass.p, nN * sizeof(double), cudaMemcpyDeviceToHost));
    s->aff_m_in.assign(s->ain.size(), 0.0);
    std::vector<double> aff_m_h(s->n_aff), aff_vol_h(s->n_aff), aff_S_h(9 * (size_t)s->n_aff),
        aff_stiff_h(s->n_aff);
    s->aff_com_h.assign(3 * (size_t)s->ain.size(), 0.0);
    s->aff_mode_h.assign(s->ain.size(), 0);
    for (int a = 0; a < s->n_aff; ++a) {
        const double* q = &mp[13 * (size_t)a];
        double vol = q[0], m = arho[a] * vol;
        if (!(vol > 0.0)) fail(ZEMA_ERR_INVALID_ARG, "affine body mesh encloses no volume (not closed / outward?)");
        double c[3] = {q[1] / m, q[2] / m, q[3] / m};
        aff_m_h[a] = m;
        s->aff_m_in[aff_perm[a]] = m;
        aff_vol_h[a] = vol;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) aff_S_h[9 * a + 3 * i + j] = q[4 + 3 * i + j] - m * c[i] * c[j];
        aff_stiff_h[a] = s->ain[aff_perm[a]].stiff;
        for (int i = 0; i < 3; ++i) s->aff_com_h[3 * aff_perm[a] + i] = c[i];
        s->aff_mode_h[aff_perm[a]] = s->ain[aff_perm[a]].mode;
    }
    std::vector<double> aff_com_dev(3 * (size_t)s->n_aff);
    for (int a = 0; a < s->n_aff; ++a)
        for (int i = 0; i < 3; ++i) aff_com_dev[3 * a + i] = s->aff_com_h[3 * aff_perm[a] + i];
    up(s, s->aff_m, aff_m_h);
    up(s, s->aff_vol, aff_vol_h);
    up(s, s->aff_S, aff_S_h);
    up(s, s->aff_stiff, aff_stiff_h);
    up(s, s->aff_com, aff_com_dev);
    // joint constants at the initial state
    {
        const int NJ = (int)s->joint_order.size();
        std::vector<JointDev> jd(NJ);
        std::vector<int> ejs(NE + 1, 0);
        auto inv3 = [](const double* M, double* I) {
            double C[9] = {M[4] * M[8] - M[5] * M[7], M[5] * M[6] - M[3] * M[8], M[3] * M[7] - M[4] * M[6],
                           M[2] * M[7] - M[1] * M[8], M[0] * M[8] - M[2] * M[6], M[1] * M[6] - M[0] * M[7],
                           M[1] * M[5] - M[2] * M[4], M[2] * M[3] - M[0] * M[5], M[0] * M[4] - M[1] * M[3]};
            const double d = M[0] * C[0] + M[1] * C[1] + M[2] * C[2];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) I[3 * i + j] = C[3 * j + i] / d;
            return d;
        };
        for (int k = 0; k < NJ; ++k) {
            const JointIn& J = s->jin[s->joint_order[k]];
            const AffIn& B1 = s->ain[J.a1];
            const AffIn& B2 = s->ain[J.a2];
            JointDev& D = jd[k];
            D.n1 = s->aff_node0_h[J.a1];
            D.n2 = s->aff_node0_h[J.a2];
            D.fix1 = B1.mode == 1;
            D.fix2 = B2.mode == 1;
            D.env = B1.env;
            D.kappa = J.kappa > 0.0 ? J.kappa : 1e3 * 0.5 * (s->aff_m_in[J.a1] + s->aff_m_in[J.a2]);
            const double* A1 = B1.q0 + 3;  // A by rows
            const double* A2 = B2.q0 + 3;
            if (!(inv3(A1, D.B1) > 0.0) || !(inv3(A2, D.B2) > 0.0))
                fail(ZEMA_ERR_INVALID_ARG, "a jointed body's initial A is not invertible with det > 0");
            // joint point: body 1's centre of mass at the initial state
            double P1[3], P2[3];
            for (int i = 0; i < 3; ++i) {
                P1[i] = B1.q0[i];
                P2[i] = B2.q0[i];
                for (int j = 0; j < 3; ++j) {
                    P1[i] += A1[3 * i + j] * s->aff_com_h[3 * J.a1 + j];
                    P2[i] += A2[3 * i + j] * s->aff_com_h[3 * J.a2 + j];
                }
            }
            for (int i = 0; i < 3; ++i) {
                D.u1[i] = 0.0;
                D.u2[i] = 0.0;
                D.d1[i] = 0.0;
                for (int j = 0; j < 3; ++j) {
                    D.u2[i] += D.B2[3 * i + j] * (P1[j] - P2[j]);
                    D.d1[i] += D.B1[3 * i + j] * J.axis[j];
                }
            }
            ejs[D.env + 1] += 1;
        }
        for (int e = 0; e < NE; ++e) ejs[e + 1] += ejs[e];
        s->joints.ensure(A, NJ + 1);
        if (NJ) ZCHECK(cudaMemcpy(s->joints.p, jd.data(), NJ * sizeof(JointDev), cudaMemcpyHostToDevice));
        up(s, s->env_joint_start, ejs);
        std::vector<double> lz(12 * (size_t)NJ + 12, 0.0);
        up(s, s->lamJ, lz);
        s->lamJ_save.ensure(A, 12 * (size_t)NJ + 12);
    }
    // surface rest positions relative to the centre of mass (affine)
    sv_x0_h.assign(3 * (size_t)s->n_sv, 0.0);
    for (int i = 0; i < s->n_sv; ++i)
        if (sv_aff_body[i] >= 0)
            for (int j = 0; j < 3; ++j) sv_x0_h[3 * i + j] = sv_rest_h[3 * i + j] - aff_com_dev[3 * sv_aff_body[i] + j];
    up(s, s->sv_x0, sv_x0_h);
    // ---- initial state: affine q (row, caller frame) -> centred columns
    for (int a = 0; a < s->n_aff; ++a) {
        AffIn& B = s->ain[aff_perm[a]];
        int n0 = aff_node0_dev[a];
        const double* c = &aff_com_dev[3 * a];
        const double* q = B.q0;
        const double* qd = B.qd0;
        for (int i = 0; i < 3; ++i) {
            double Ac = q[3 + 3 * i] * c[0] + q[4 + 3 * i] * c[1] + q[5 + 3 * i] * c[2];
            double Adc = qd[3 + 3 * i] * c[0] + qd[4 + 3 * i] * c[1] + qd[5 + 3 * i] * c[2];
            x_h[3 * n0 + i] = q[i] + Ac;
            v_h[3 * n0 + i] = B.mode == 1 ? 0.0 : qd[i] + Adc;
            for (int k = 0; k < 3; ++k) {
                x_h[3 * (n0 + 1 + k) + i] = q[3 + 3 * i + k];
                v_h[3 * (n0 + 1 + k) + i] = B.mode == 1 ? 0.0 : qd[3 + 3 * i + k];
            }
        }
    }
    up(s, s->x, x_h);
    up(s, s->v, v_h);
    // kinematic targets default to q0, multipliers to 0
    std::vector<double> qt_h(12 * (size_t)s->n_aff + 12, 0.0), lam_h(12 * (size_t)s->n_aff + 12, 0.0);
    for (int a = 0; a < s->n_aff; ++a)
        for (int k = 0; k < 12; ++k) qt_h[12 * a + k] = s->ain[aff_perm[a]].q0[k];
    up(s, s->qtarget, qt_h);
    up(s, s->lamA, lam_h);
    up(s, s->lamA_prev, lam_h);
    // ---- per-env bbox diagonal (and centre) of the initial state
    s->diag_h.assign(NE, 0.0);
    std::vector<double> envc_h(3 * (size_t)NE, 0.0);
    for (int e = 0; e < NE; ++e) {
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        auto acc = [&](const double* p) {
            for (int j = 0; j < 3; ++j) {
                lo[j] = std::min(lo[j], p[j]);
                hi[j] = std::max(hi[j], p[j]);
            }
        };
        for (size_t i = 0; i < s->tin.size(); ++i)
            if (s->tin[i].env == e)
                for (size_t k = 0; k < s->tin[i].x0.size() / 3; ++k) acc(&s->tin[i].x0[3 * k]);
        for (size_t i = 0; i < s->ain.size(); ++i)
            if (s->ain[i].env == e) {
                const AffIn& B = s->ain[i];
                for (size_t k = 0; k < B.V.size() / 3; ++k) {
                    double w[3];
                    for (int r = 0; r < 3; ++r)
                        w[r] = B.q0[r] + B.q0[3 + 3 * r] * B.V[3 * k] + B.q0[4 + 3 * r] * B.V[3 * k + 1] +
                               B.q0[5 + 3 * r] * B.V[3 * k + 2];
                    acc(w);
                }
            }
        double d2 = 0.0;
        for (int j = 0; j < 3; ++j) {
            d2 += (hi[j] - lo[j]) * (hi[j] - lo[j]);
            envc_h[3 * e + j] = 0.5 * (lo[j] + hi[j]);
        }
        s->diag_h[e] = std::sqrt(d2);
    }
    s->tol_h.assign(NE, 0.0);
    for (int e = 0; e < NE; ++e) s->tol_h[e] = s->P.newton_tol_rel * s->diag_h[e] * s->P.dt;
    up(s, s->tolv, s->tol_h);
    // ---- state buffers
    size_t n3 = 3 * (size_t)nN + 3;
    for (DBuf<double>* b : {&s->xt, &s->xhat, &s->p, &s->xtrial, &s->g, &s->b, &s->r, &s->z, &s->pp, &s->q})
        b->ensure(A, n3);
    for (DBuf<double>* b : {&s->X, &s->Xt, &s->X1}) b->ensure(A, 3 * (size_t)s->n_sv + 3);
    s->stage_blk.ensure(A, 144 * ((size_t)s->n_tets + s->n_aff) + 576 * s->jin.size() + 9);
    s->stage_g.ensure(A, 12 * (size_t)s->n_tets + 12);
    s->S_val.ensure(A, 9 * (size_t)s->n_sblocks + 9);
    s->Minv_s.ensure(A, 9 * (size_t)nN + 9);
    s->Minv_a.ensure(A, 144 * (size_t)s->n_aff + 144);
    for (DBuf<double>* b : {&s->kappa, &s->kappa_min, &s->alpha, &s->E, &s->dmin, &s->tol2_env}) b->ensure(A, NE + 1);
    for (DBuf<double>* b : {&s->part, &s->part2, &s->part3, &s->part4, &s->part5, &s->part6, &s->part7})
        b->ensure(A, (size_t)ET_COUNT * NE * kChunks + 8);
    for (DBuf<int>* b : {&s->conv, &s->pcg_iters, &s->need, &s->skip, &s->pcg_refines, &s->ls_skip})
        b->ensure(A, NE + 1);
    s->capflag.ensure(A, 1);
    for (DBuf<uint32_t>* b : {&s->pt_env, &s->ee_env, &s->m_env, &s->act_env, &s->swept_env, &s->lag_env})
        b->ensure(A, NE + 2);
    if (!s->h32) ZCHECK(cudaMallocHost(&s->h32, 64 * sizeof(uint32_t)));
    if (!s->hd) ZCHECK(cudaMallocHost(&s->hd, (8 * (size_t)NE + 64) * sizeof(double)));
    if (!s->hi) ZCHECK(cudaMallocHost(&s->hi, (4 * (size_t)NE + 64) * sizeof(int)));
    if (!s->h_alpha) ZCHECK(cudaMallocHost(&s->h_alpha, ((size_t)NE + 8) * sizeof(double)));
    if (!s->h_up_i) ZCHECK(cudaMallocHost(&s->h_up_i, (size_t)kUpSlots * NE * sizeof(int)));
    if (!s->h_up_d) ZCHECK(cudaMallocHost(&s->h_up_d, (size_t)kUpSlots * NE * sizeof(double)));
    if (!s->h_pcg) ZCHECK(cudaMallocHost(&s->h_pcg, (3 * (size_t)NE + 8) * sizeof(int)));
    // learned warm start: soft vertices in node order, their body, per-body
    // node range and rest half-diagonal
    {
        std::vector<int> tb0, tbn, node_tb(nN, -1);
        std::vector<double> tbR;
        for (size_t b = 0; b < s->tin.size(); ++b) {
            const int n0 = s->tet_body_node0[b], nv = (int)(s->tin[b].X.size() / 3);
            tb0.push_back(n0);
            tbn.push_back(nv);
            double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int k = 0; k < nv; ++k)
                for (int j = 0; j < 3; ++j) {
                    lo[j] = std::min(lo[j], s->tin[b].X[3 * k + j]);
                    hi[j] = std::max(hi[j], s->tin[b].X[3 * k + j]);
                }
            double d2 = 0.0;
            for (int j = 0; j < 3; ++j) d2 += (hi[j] - lo[j]) * (hi[j] - lo[j]);
            tbR.push_back(std::max(0.5 * std::sqrt(d2), 1e-12));
            for (int k = 0; k < nv; ++k) node_tb[n0 + k] = (int)b;
        }
        std::vector<int> soft, sbody;
        for (int n = 0; n < nN; ++n)
            if (node_tb[n] >= 0) {
                soft.push_back(n);
                sbody.push_back(node_tb[n]);
            }
        s->ws_ns = (int)soft.size();
        s->ws_nb = (int)tb0.size();
        up(s, s->ws_soft, soft);
        up(s, s->ws_body, sbody);
        up(s, s->tb_node0, tb0);
        up(s, s->tb_nv, tbn);
        up(s, s->tb_R, tbR);
        s->tb_c.ensure(A, 3 * (size_t)s->ws_nb + 3);
        s->ws_best.ensure(A, (size_t)nN + 1);
        s->ws_feat.ensure(A, (size_t)kWsFeatures * s->ws_ns + kWsFeatures);
        s->ws_out.ensure(A, (size_t)kWsOutputs * s->ws_ns + kWsOutputs);
        // dynamic affine bodies for the per-body network
        std::vector<int> aff;
        std::vector<double> aR, envd(s->diag_h);
        for (int a = 0; a < s->n_aff; ++a) {
            const AffIn& B = s->ain[aff_perm[a]];
            if (B.mode != 0) continue;
            double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (size_t k = 0; k < B.V.size() / 3; ++k)
                for (int j = 0; j < 3; ++j) {
                    lo[j] = std::min(lo[j], B.V[3 * k + j]);
                    hi[j] = std::max(hi[j], B.V[3 * k + j]);
                }
            double d2 = 0.0;
            for (int j = 0; j < 3; ++j) d2 += (hi[j] - lo[j]) * (hi[j] - lo[j]);
            aff.push_back(a);
            aR.push_back(std::max(0.5 * std::sqrt(d2), 1e-12));
        }
        for (double& d : envd) d = std::max(d, 1e-12);
        s->ws_na = (int)aff.size();
        up(s, s->ws_aff, aff);
        up(s, s->ws_aR, aR);
        up(s, s->ws_envc, envc_h);
        up(s, s->ws_envd, envd);
        s->ws_afeat.ensure(A, (size_t)kWsAffFeatures * s->ws_na + kWsAffFeatures);
        s->ws_aout.ensure(A, (size_t)kWsAffOutputs * s->ws_na + kWsAffOutputs);
    }
    // kappa: user value or pending rule
    std::vector<double> kap(NE, s->P.kappa > 0 ? s->P.kappa : 0.0);
    up(s, s->kappa, kap);
    up(s, s->kappa_min, kap);
    s->kappa_ready.assign(NE, s->P.kappa > 0 ? 1 : 0);
    // ---- Geo view
    Geo& G = s->G;
    G.n_nodes = nN;
    G.n_soft = 0;
    G.n_aff = s->n_aff;
    G.n_tets = s->n_tets;
    G.n_sv = s->n_sv;
    G.n_edges = s->n_edges;
    G.n_tris = s->n_tris;
    G.n_envs = NE;
    G.n_units = s->n_units;
    G.n_bodies = (int)s->bodies.size();
    G.h = s->P.dt;
    G.dhat = s->P.dhat;
    G.eps_v = s->P.eps_v;
    G.node_env = s->node_env.p;
    G.node_fixed = s->node_fixed.p;
    G.node_mass = s->node_mass.p;
    G.env_node_start = s->env_node_start.p;
    G.tets = s->tets.p;
    G.Dminv = s->Dminv.p;
    G.tvol = s->tvol.p;
    G.tmu = s->tmu.p;
    G.tlam = s->tlam.p;
    G.tmodel = s->tmodel.p;
    G.spring_k = s->has_springs ? s->spring_k.p : nullptr;
    G.spring_x = s->spring_x.p;
    G.env_tet_start = s->env_tet_start.p;
    G.aff_node0 = s->aff_node0.p;
    G.aff_mode = s->aff_mode.p;
    G.aff_m = s->aff_m.p;
    G.aff_S = s->aff_S.p;
    G.aff_vol = s->aff_vol.p;
    G.aff_stiff = s->aff_stiff.p;
    G.aff_com = s->aff_com.p;
    G.env_aff_start = s->env_aff_start.p;
    G.n_joints = (int)s->joint_order.size();
    G.joints = s->joints.p;
    G.env_joint_start = s->env_joint_start.p;
    G.lamJ = s->lamJ.p;
    G.unit_kind = s->unit_kind.p;
    G.unit_idx = s->unit_idx.p;
    G.env_unit_start = s->env_unit_start.p;
    G.sv_node = s->sv_node.p;
    G.sv_aff = s->sv_aff.p;
    G.sv_x0 = s->sv_x0.p;
    G.sv_rest = s->sv_rest.p;
    G.sv_body = s->sv_body.p;
    G.sv_env = s->sv_env.p;
    G.body_class = s->body_class.p;
    G.body_mu = s->body_mu.p;
    G.edges = s->edges.p;
    G.tris = s->tris.p;
    G.edge_rest2 = s->edge_rest2.p;
    G.env_sv_start = s->env_sv_start.p;
    G.env_edge_start = s->env_edge_start.p;
    G.node_tet_ptr = s->node_tet_ptr.p;
    G.node_tet_idx = s->node_tet_idx.p;
    G.S_rowptr = s->S_rowptr.p;
    G.S_col = s->S_col.p;
    G.S_src_ptr = s->S_src_ptr.p;
    G.S_src = s->S_src.p;
    // dynamic shared memory opt-in for the per-thread matrix kernels
    ZCHECK(cudaFuncSetAttribute(k_elastic_gh<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 81 * EL_T * 8));
    ZCHECK(cudaFuncSetAttribute(k_elastic_gh<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 81 * EL_T * 4));
    ZCHECK(cudaStreamSynchronize(st));
    for (size_t b = 0; b < s->tin.size(); ++b)
        if (!s->tin[b].spring_v.empty()) upload_springs(s, (int)b);
    s->finalized = true;
}

// ---------------------------------------------------------------------------
// Pair lists
// ---------------------------------------------------------------------------
// Broad phase over X0 (-> X1) and merge into env-ordered PairRec `out` with
// env offsets; returns the count.
__global__ void k_reset_dmin(double* dmin, int n, const int* keep) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n && !(keep && keep[e])) dmin[e] = INFINITY;
}

// Candidate pairs (static boxes of X0, or swept X0 -> X1) into `out` with
// per-env offsets.  Only the primitives of envs e_lo..e_hi are searched (the
// envs outside that range contribute no pairs; e_hi < e_lo searches nothing),
// so that a batch whose last few envs still iterate searches only their
// range; inside it, envs flagged in env_skip contribute no pairs.
uint32_t candidates(zema_scene* s, const double* X0, const double* X1, DBuf<PairRec>& out, DBuf<uint32_t>& env_off,
                    const int* env_skip = nullptr, int e_lo = 0, int e_hi = -2) {
    cudaStream_t st = s->st;
    if (e_hi == -2) e_hi = s->n_envs - 1;
    BPView v;
    // an empty range searches nothing (all offsets 0)
    const bool empty = e_hi < e_lo;
    const int sv0 = empty ? 0 : s->env_sv_start_h[e_lo], sv1 = empty ? 0 : s->env_sv_start_h[e_hi + 1];
    const int ed0 = empty ? 0 : s->env_edge_start_h[e_lo], ed1 = empty ? 0 : s->env_edge_start_h[e_hi + 1];
    const int tr0 = empty ? 0 : s->env_tri_start_h[e_lo], tr1 = empty ? 0 : s->env_tri_start_h[e_hi + 1];
    v.nsv = sv1 - sv0;
    v.ne = ed1 - ed0;
    v.nt = tr1 - tr0;
    v.sv_base = sv0;
    v.edge_base = ed0;
    v.tri_base = tr0;
    v.X0 = X0;
    v.X1 = X1;
    v.sv_body = s->sv_body.p;
    v.body_class = s->body_class.p;
    v.sv_env = s->sv_env.p;
    v.edges = s->edges.p;
    v.tris = s->tris.p;
    v.infl = 0.5 * s->P.dhat;
    v.inv_cell = 1.0 / s->cell;
    v.env_skip = env_skip;
    v.env_tri_start = s->env_tri_start.p;
    v.env_edge_start = s->env_edge_start.p;
    s->bp.run(&s->A, v, st);
    uint32_t n = s->bp.n_pt + s->bp.n_ee;
    out.ensure(&s->A, n + 1);
    int NE = s->n_envs;
    ZL(k_pair_env_offsets, div_up(NE + 1, 64), 64, 0, st)(s->G, s->bp.qoff_pt.p, s->bp.qoff_ee.p, v.sv_base, v.nsv,
                                                          v.edge_base, v.ne, s->pt_env.p, s->ee_env.p, env_off.p);
    ZLAUNCH();
    if (n)
        ZL(k_merge_pairs, div_up(n, TB), TB, 0, st)(s->G, s->bp.pt.p, s->bp.ee.p, s->pt_env.p, s->ee_env.p, env_off.p,
                                                   (int)n, out.p);
    ZLAUNCH();
    s->S.max_candidates = std::max<int64_t>(s->S.max_candidates, n);
    return n;
}

// The first and last env not flagged in done (e_hi < e_lo when all are)
void active_range(const std::vector<int>& done, int& e_lo, int& e_hi) {
    const int NE = (int)done.size();
    e_lo = 0;
    while (e_lo < NE && done[e_lo]) ++e_lo;
    e_hi = NE - 1;
    while (e_hi >= e_lo && done[e_hi]) --e_hi;
}

// Active pairs (d < dhat) at X among the n pairs of `list` (env offsets
// `list_env`): fills s->act / s->act_env and, if asked, the per-env minimum
// distance of active pairs.
uint32_t active_from(zema_scene* s, const double* X, const PairRec* list, const uint32_t* list_env, uint32_t n,
                     bool want_dmin, const int* dmin_keep = nullptr) {
    cudaStream_t st = s->st;
    int NE = s->n_envs;
    if (want_dmin) {
        // d_min restarts at infinity except for envs flagged in dmin_keep
        // (converged envs whose pairs the list no longer holds)
        ZL(k_reset_dmin, div_up(NE, 64), 64, 0, st)(s->dmin.p, NE, dmin_keep);
        ZLAUNCH();
    }
    s->flag.ensure(&s->A, n + 1);
    s->flagoff.ensure(&s->A, n + 2);
    s->tmp32.ensure(&s->A, scan_tmp_size(n + 1));
    if (n)
        ZL(k_active_flags, div_up(n, TB), TB, 0, st)(s->G, X, list, (int)n, s->flag.p, want_dmin ? s->dmin.p : nullptr);
    ZLAUNCH();
    exclusive_scan(s->flag.p, s->flagoff.p, n, s->tmp32.p, st);
    ZCHECK(cudaMemcpyAsync(s->h32, s->flagoff.p + n, 4, cudaMemcpyDeviceToHost, st));
    ZL(k_env_gather, div_up(NE + 1, 64), 64, 0, st)(s->flagoff.p, list_env, NE, s->act_env.p);
    ZLAUNCH();
    ZCHECK(cudaStreamSynchronize(st));
    uint32_t na = s->h32[0];
    s->act.ensure(&s->A, na + 1);
    if (n) ZL(k_compact_pairs, div_up(n, TB), TB, 0, st)(list, s->flag.p, s->flagoff.p, (int)n, s->act.p);
    ZLAUNCH();
    s->n_act = na;
    s->S.max_active = std::max<int64_t>(s->S.max_active, na);
    return na;
}

// active pairs of X from a fresh broad phase over X
uint32_t active_pairs(zema_scene* s, const double* X, bool want_dmin) {
    uint32_t n = candidates(s, X, nullptr, s->cand, s->m_env);
    return active_from(s, X, s->cand.p, s->m_env.p, n, want_dmin);
}

// ---------------------------------------------------------------------------
// Energies
// ---------------------------------------------------------------------------
AffKin kin(zema_scene* s) { return AffKin{s->qtarget.p, s->lamA.p}; }

Lag lagv(zema_scene* s) {
    return Lag{s->lag.p, s->lag_w.p, s->lag_n.p, s->lag_c.p, s->lag_env.p, (int)s->n_lag};
}

// Per-env incremental potential at node positions xe (barrier over the pairs
// in `pairs` with env offsets `poff`); result in s->hd[0..NE).
void energy(zema_scene* s, const double* xe, const PairRec* pairs, const uint32_t* poff, bool barrier = true,
            bool friction = true) {
    cudaStream_t st = s->st;
    int NE = s->n_envs;
    ZCHECK(cudaMemsetAsync(s->part.p, 0, (size_t)ET_COUNT * NE * kChunks * sizeof(double), st));
    ZL(k_sv_pos, div_up(s->n_sv, TB), TB, 0, st)(s->G, xe, s->X1.p);
    ZL(k_soft_energy, red_grid(NE), kRedThreads, 0, st)(s->G, xe, s->xhat.p, s->part.p);
    ZL(k_affine_energy, red_grid(NE), kRedThreads, 0, st)(s->G, xe, s->xhat.p, kin(s), s->part.p);
    if (barrier && pairs)
        ZL(k_barrier_energy, red_grid(NE), kRedThreads, 0, st)(s->G, s->X1.p, pairs, poff, s->kappa.p, s->part.p);
    if (friction && s->n_lag)
        ZL(k_friction_energy, red_grid(NE), kRedThreads, 0, st)(s->G, s->X1.p, s->Xt.p, lagv(s), s->part.p);
    if (s->G.n_joints) ZL(k_joint_energy, red_grid(NE), kRedThreads, 0, st)(s->G, xe, s->part.p);
    ZL(k_energy_total, div_up(NE, 64), 64, 0, st)(s->part.p, ET_COUNT, NE, s->E.p);
    ZLAUNCH();
    ZCHECK(cudaMemcpyAsync(s->hd, s->E.p, NE * sizeof(double), cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------------------
// Gradient and Hessian assembly at x; g and the BSR (S, C) are filled.
// ---------------------------------------------------------------------------
// Hessian blocks, staging, BSR values and preconditioner in T (double: FP64
// path; float: mixed path), gradients always FP64.
template <class T>
void grad_hess_t(zema_scene* s, bool barrier, bool friction, bool hess) {
    cudaStream_t st = s->st;
    T* stage = (T*)s->stage_blk.p;
    T* S_val = (T*)s->S_val.p;
    Geo& G = s->G;
    Allocator* A = &s->A;
    // per tet: indices 16 B, Dm^-1 72 B, volume and Lame 24 B, positions 96 B
    // in; 16 blocks 1152 B and gradient 96 B out
    alg_bytes_hint(1456.0 * s->n_tets);
    if (s->n_tets)
        ZL(k_elastic_gh<T>, div_up(s->n_tets, EL_T), EL_T, 81 * EL_T * sizeof(T), st)(G, s->x.p, stage, s->stage_g.p);
    ZLAUNCH();
    ZCHECK(cudaMemsetAsync(s->g.p, 0, 3 * (size_t)s->n_nodes * sizeof(double), st));
    if (s->n_aff)
        ZL(k_affine_gh<T>, div_up(s->n_aff, kAffBodies), kCoopLanes * kAffBodies, 0, st)(
            G, s->x.p, s->xhat.p, kin(s), stage + 144 * (size_t)s->n_tets, s->g.p);
    ZLAUNCH();
    ZL(k_soft_grad, div_up(s->n_nodes, TB), TB, 0, st)(G, s->x.p, s->xhat.p, s->stage_g.p, s->g.p);
    ZLAUNCH();
    if (G.n_joints) {
        ZL(k_joint_gh<T>, 1, 32, 0, st)(G, s->x.p, stage + 144 * ((size_t)s->n_tets + s->n_aff), s->g.p);
        ZLAUNCH();
    }
    if (hess) {
        ZL(k_static_values<T>, div_up(s->n_sblocks, TB), TB, 0, st)(G, s->n_sblocks, stage, S_val);
        ZL(k_static_diag<T>, div_up(s->n_nodes, TB), TB, 0, st)(G, s->S_diag.p, S_val);
        ZLAUNCH();
    }
    // contact records: active barrier pairs then lagged friction pairs
    uint32_t na = barrier ? s->n_act : 0, nl = friction ? s->n_lag : 0;
    uint32_t nr = na + nl;
    s->pH.ensure(A, 144 * (size_t)nr + 144);
    s->pG.ensure(A, 12 * (size_t)nr + 12);
    T* pH = (T*)s->pH.p;
    if (na) {
        // few pairs: a half-warp per pair keeps many warps busy; many pairs:
        // 32 per warp issues the FP64 part once per 32 pairs
        if (na >= (uint32_t)kSplitMinPairs) {
            s->pflag.ensure(A, na + 1);
            ZL(k_barrier_gh_raw<T>, div_up(na, kRawThreads), kRawThreads, 0, st)(G, s->X.p, s->act.p, (int)na,
                                                                               s->kappa.p, pH, s->pG.p, s->pflag.p);
            ZL(k_barrier_project<T>, div_up(na, kProjPairs), kCoopLanes * kProjPairs, 0, st)(
                G, s->act.p, (int)na, s->kappa.p, s->pflag.p, pH);
        } else
            ZL(k_barrier_gh_half<T>, div_up(na, kCoopPairs), kCoopLanes * kCoopPairs, 0, st)(
                G, s->X.p, s->act.p, (int)na, s->kappa.p, pH, s->pG.p);
    }
    if (nl)
        ZL(k_friction_gh<T>, div_up(nl, 128), 128, 0, st)(G, s->X.p, s->Xt.p, lagv(s), pH + 144 * (size_t)na,
                                                           s->pG.p + 12 * (size_t)na);
    ZLAUNCH();
    // one record list: act then lag
    DBuf<PairRec>& recs = s->recs;
    recs.ensure(A, nr + 1);
    if (na) ZCHECK(cudaMemcpyAsync(recs.p, s->act.p, na * sizeof(PairRec), cudaMemcpyDeviceToDevice, st));
    if (nl) ZCHECK(cudaMemcpyAsync(recs.p + na, s->lag.p, nl * sizeof(PairRec), cudaMemcpyDeviceToDevice, st));
    s->C_rowptr.ensure(A, s->n_nodes + 2);
    if (nr == 0) {
        ZCHECK(cudaMemsetAsync(s->C_rowptr.p, 0, (s->n_nodes + 1) * sizeof(int), st));
        s->n_cblocks = 0;
        s->n_cblocks_pending = false;
        s->C_col.ensure(A, 1);
        s->C_val.ensure(A, 9);
        return;
    }
    s->cnt_blk.ensure(A, nr + 1);
    s->off_blk.ensure(A, nr + 2);
    s->cnt_g.ensure(A, nr + 1);
    s->off_g.ensure(A, nr + 2);
    ZL(k_contact_count, div_up(nr, TB), TB, 0, st)(G, recs.p, (int)nr, s->cnt_blk.p, s->cnt_g.p);
    ZLAUNCH();
    s->tmp32.ensure(A, scan_tmp_size(nr + 1));
    exclusive_scan(s->cnt_blk.p, s->off_blk.p, nr, s->tmp32.p, st);
    exclusive_scan(s->cnt_g.p, s->off_g.p, nr, s->tmp32.p, st);
    ZCHECK(cudaMemcpyAsync(s->h32, s->off_blk.p + nr, 4, cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaMemcpyAsync(s->h32 + 1, s->off_g.p + nr, 4, cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaStreamSynchronize(st));
    uint32_t nb = s->h32[0], ng = s->h32[1];
    s->bkey.ensure(A, nb + 1);
    s->bkey2.ensure(A, nb + 1);
    s->bval.ensure(A, nb + 1);
    s->bval2.ensure(A, nb + 1);
    s->bstage.ensure(A, 9 * (size_t)nb + 9);
    s->gkey.ensure(A, ng + 1);
    s->gkey2.ensure(A, ng + 1);
    s->gval.ensure(A, ng + 1);
    s->gval2.ensure(A, ng + 1);
    s->gstage.ensure(A, 3 * (size_t)ng + 3);
    ZL(k_contact_emit<T>, div_up((long long)nr * kEmitPairLanes, 128), 128, 0, st)(G, recs.p, (int)nr, pH, s->pG.p, s->off_blk.p, s->off_g.p,
                                                        s->bkey.p, s->bval.p, (T*)s->bstage.p, s->gkey.p, s->gval.p,
                                                        s->gstage.p);
    ZLAUNCH();
    int nbits_node = 1;
    while ((1ll << nbits_node) < (long long)s->n_nodes) ++nbits_node;
    uint32_t mx = std::max(nb, ng) + 2;
    s->tmp32.ensure(A, std::max(radix_tmp_size(mx), scan_tmp_size(mx)));
    radix_sort(s->bkey.p, s->bval.p, s->bkey2.p, s->bval2.p, nb, 2 * nbits_node, s->tmp32.p, st);
    radix_sort(s->gkey.p, s->gval.p, s->gkey2.p, s->gval2.p, ng, nbits_node, s->tmp32.p, st);
    // unique blocks
    s->head.ensure(A, mx);
    s->hoff.ensure(A, mx + 1);
    s->seg.ensure(A, mx + 1);
    s->ukey.ensure(A, mx);
    // the unique counts stay on the device: the unique-block and unique-node
    // launches read them there (sized by their upper bounds nb and ng), and
    // the host picks the block count up at the solve's next read-back
    s->cnt_u.ensure(A, 4);
    ZL(k_heads, div_up(nb, TB), TB, 0, st)(s->bkey.p, nb, s->head.p);
    exclusive_scan(s->head.p, s->hoff.p, nb, s->tmp32.p, st);
    ZL(k_seg_starts, div_up(nb + 1, TB), TB, 0, st)(s->head.p, s->hoff.p, nb, s->seg.p);
    ZCHECK(cudaMemcpyAsync(s->cnt_u.p, s->hoff.p + nb, 4, cudaMemcpyDeviceToDevice, st));
    ZCHECK(cudaMemcpyAsync(s->h32 + 8, s->hoff.p + nb, 4, cudaMemcpyDeviceToHost, st));
    s->C_val.ensure(A, 9 * (size_t)nb + 9);
    s->C_col.ensure(A, nb + 1);
    const int seg_grid = std::max(1, std::min(div_up(32 * (long long)nb, 128), 148 * 32));
    ZL((k_seg_sum<9, T>), seg_grid, 128, 0, st)(s->seg.p, s->cnt_u.p, s->bval.p, (const T*)s->bstage.p,
                                               (T*)s->C_val.p, s->bkey.p, s->ukey.p);
    ZL(k_contact_rows, div_up(s->n_nodes + 1, TB), TB, 0, st)(s->ukey.p, s->cnt_u.p, s->n_nodes, s->C_rowptr.p,
                                                             s->C_col.p);
    ZLAUNCH();
    s->n_cblocks_pending = true;
    // unique gradient nodes
    ZL(k_heads, div_up(ng, TB), TB, 0, st)(s->gkey.p, ng, s->head.p);
    exclusive_scan(s->head.p, s->hoff.p, ng, s->tmp32.p, st);
    ZL(k_seg_starts, div_up(ng + 1, TB), TB, 0, st)(s->head.p, s->hoff.p, ng, s->seg.p);
    ZCHECK(cudaMemcpyAsync(s->cnt_u.p + 1, s->hoff.p + ng, 4, cudaMemcpyDeviceToDevice, st));
    s->gsum.ensure(A, 3 * (size_t)ng + 3);
    const int gseg_grid = std::max(1, std::min(div_up(32 * (long long)ng, 128), 148 * 32));
    ZL((k_seg_sum<3, double>), gseg_grid, 128, 0, st)(s->seg.p, s->cnt_u.p + 1, s->gval.p, s->gstage.p, s->gsum.p,
                                                      s->gkey.p, s->ukey.p);
    ZL(k_add_contact_grad, div_up(ng, 128), 128, 0, st)(s->ukey.p, s->gsum.p, s->cnt_u.p + 1, s->g.p);
    ZLAUNCH();
}

void grad_hess(zema_scene* s, bool barrier = true, bool friction = true, bool hess = true) {
    if (s->P.precision == 1)
        grad_hess_t<float>(s, barrier, friction, hess);
    else
        grad_hess_t<double>(s, barrier, friction, hess);
}

// ---------------------------------------------------------------------------
// Cluster PCG configuration: CTAs per env ~ one per 128 nodes (at most 16,
// the largest cluster the device accepts), shared memory for the staged env
// vector, the owned rows' q and the affine rows' partials.
// ---------------------------------------------------------------------------
constexpr size_t kPcgcMaxSmem = 200 * 1024;
// dynamic shared memory of the variant with two CTAs per SM
constexpr size_t kPcgcMaxSmem2 = 96 * 1024;

// A cluster schedule code: CTAs per env (1..16), plus 100 for the variant
// that keeps two CTAs resident per SM; plus 1000 for the size-binned form,
// where the low digits are a multiplier m (1 or 2) and every env runs with
// m times the smallest cluster whose CTAs hold its rows (at most 16), one
// launch per cluster size.
inline bool sched_binned(int code) { return code >= 1000; }
inline int sched_cs(int code) { return code % 100; }
inline int sched_occ(int code) { return (code % 1000) >= 100 ? 2 : 1; }
template <class T>
inline auto pcgc_kernel(int code) {
    return sched_occ(code) == 2 ? k_pcg_cluster<T, 2> : k_pcg_cluster<T, 1>;
}

// rows a CTA may own (the solve balances rows by their blocks within this
// bound): twice the equal share, at most what its threads hold in registers
int pcgc_max_rows(const zema_scene* s, int code) {
    if (sched_binned(code)) return kPcgcOwn * kPcgcThreads + 1;  // every group's bound
    const int cs = sched_cs(code);
    return std::min(2 * ((s->pcgc_max_soft + cs - 1) / cs) + 1, kPcgcOwn * kPcgcThreads + 1);
}

// SpMV chunks a CTA can hold (0: one task per row; chunking measured slower
// on the grasp workloads, so it is off)
int pcgc_chunk_cap(const zema_scene*, int) { return 0; }

template <class T>
size_t pcgc_smem_base(const zema_scene* s, int code) {
    const size_t tasks = (size_t)pcgc_max_rows(s, code) + 4 * (size_t)s->pcgc_max_aff, ch = pcgc_chunk_cap(s, code);
    return (tasks + ch) * sizeof(int4) + ((tasks + 4) & ~(size_t)3) * sizeof(int) +
           (3 * (kPcgcThreads / 32) + 8 + pcgc_pstride<T>() * (size_t)s->pcgc_max_env_nodes +
            3 * (size_t)pcgc_max_rows(s, code) + 24 * (size_t)s->pcgc_max_aff + 3 * ch) *
               sizeof(T) +
           16;  // alignment of the staged slice
}

// Blocks of a CTA's matrix slice that the solve may stage in shared memory:
// all the space left under the budget, when that holds the largest static
// slice (soft rows' S blocks and the CTA's share of the affine rows') with
// room for contact blocks; 0 (the solve reads the matrix from L1/L2) if not.
template <class T>
int pcgc_slice_cap(const zema_scene* cs_scene, int code) {
    zema_scene* s = const_cast<zema_scene*>(cs_scene);
    const auto key = std::make_pair((int)sizeof(T), code);
    auto hit = s->pcgc_cap.find(key);
    if (hit != s->pcgc_cap.end()) return hit->second;
    const int cs = sched_cs(code);
    if (sizeof(T) != sizeof(float) || sched_occ(code) == 2 || sched_binned(code)) {  // staged: FP32, one per SM, uniform
        s->pcgc_cap[key] = 0;
        return 0;
    }
    const std::vector<int>& rp = s->S_rowptr_h;
    long long mx = 0;
    for (int e = 0; e < s->n_envs; ++e) {
        const int nb = s->env_node_start_h[e], nend = s->env_node_start_h[e + 1];
        const int ns1 = nend - 4 * (s->env_aff_start_h[e + 1] - s->env_aff_start_h[e]);
        const int n_soft = ns1 - nb;
        for (int r = 0; r < cs; ++r) {
            const int lo = nb + (int)(((long long)n_soft * r) / cs), hi = nb + (int)(((long long)n_soft * (r + 1)) / cs);
            long long c = rp[hi] - rp[lo];
            for (int n = ns1; n < nend; ++n) {
                const long long len = rp[n + 1] - rp[n];
                c += (len * (r + 1)) / cs - (len * r) / cs;
            }
            mx = std::max(mx, c);
        }
    }
    const size_t per = 12 * sizeof(float);  // a block: 9 values, its column, 2 pad
    const size_t base = pcgc_smem_base<T>(s, code);
    const long long avail = base >= kPcgcMaxSmem ? 0 : (long long)((kPcgcMaxSmem - base) / per);
    const int cap = avail >= mx + mx / 4 + 128 ? (int)avail : 0;
    s->pcgc_cap[key] = cap;
    return cap;
}

template <class T>
size_t pcgc_smem(const zema_scene* s, int code) {
    return pcgc_smem_base<T>(s, code) + (size_t)pcgc_slice_cap<T>(s, code) * 12 * sizeof(float);
}

// The env groups of a size-binned schedule with multiplier m (built once):
// env e runs with cs_e = min(16, m * c_e) CTAs, c_e the smallest power of two
// whose CTAs hold the env's soft rows; groups by cs in the order 1, 2, 4,
// 8, 16.  Returns the 6 group offsets into s->pcgc_bin_list[m].
const std::vector<int>& pcgc_bins(zema_scene* s, int m) {
    std::vector<int>& off = s->pcgc_bin_off[m];
    if (!off.empty()) return off;
    std::vector<int> grp[5];
    for (int e = 0; e < s->n_envs; ++e) {
        int c = 1;
        while (c < 16 && (s->env_soft_h[e] + c - 1) / c > kPcgcOwn * kPcgcThreads) c *= 2;
        int k = 0;
        for (int cs = std::min(16, m * c); cs > 1; cs /= 2) ++k;
        grp[k].push_back(e);
    }
    std::vector<int> list;
    off.push_back(0);
    for (int k = 0; k < 5; ++k) {
        list.insert(list.end(), grp[k].begin(), grp[k].end());
        off.push_back((int)list.size());
    }
    up(s, s->pcgc_bin_list[m], list);
    return off;
}

template <class T>
void pcgc_config(const zema_scene* s, int code, cudaLaunchConfig_t& cfg, cudaLaunchAttribute* at, int cs_group = 0,
                 int n_group = 0) {
    const int cs = cs_group ? cs_group : sched_cs(code);
    cfg.gridDim = dim3((unsigned)(cs * (cs_group ? n_group : s->n_envs)));
    cfg.blockDim = dim3(kPcgcThreads);
    cfg.dynamicSmemBytes = pcgc_smem<T>(s, code);
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
}

// CTAs per env for the cluster solve, or -1 when it cannot run (env vector
// too large for shared memory, no cluster launch on this device).
template <class T>
int pcgc_choose(zema_scene* s) {
    int want = std::min(16, std::max(1, (s->pcgc_max_env_nodes + 127) / 128));
    // the env's vector must fit in shared memory, a CTA's rows in its
    // threads' registers, the affine rows in one CTA
    if (pcgc_smem_base<T>(s, 16) > kPcgcMaxSmem || 12 * s->pcgc_max_aff > kPcgcThreads) return -1;
    ZCHECK(cudaFuncSetAttribute(k_pcg_cluster<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPcgcMaxSmem));
    ZCHECK(cudaFuncSetAttribute(k_pcg_cluster<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPcgcMaxSmem2));
    // the rest of the SM's storage stays L1 for the matrix rows (one CTA per
    // SM) or holds two CTAs' shared memory
    bool nonportable = true;
    if (cudaFuncSetAttribute(k_pcg_cluster<T, 1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(k_pcg_cluster<T, 2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        nonportable = false;
    }
    if (want > 8 && !nonportable) want = 8;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    pcgc_config<T>(s, want, cfg, at);
    int maxcs = 0;
    if (cudaOccupancyMaxPotentialClusterSize(&maxcs, k_pcg_cluster<T, 1>, &cfg) != cudaSuccess || maxcs < 1) {
        cudaGetLastError();
        return -1;
    }
    int cs = std::min(want, maxcs);
    if ((s->pcgc_max_soft + cs - 1) / cs > kPcgcOwn * kPcgcThreads || pcgc_smem<T>(s, cs) > kPcgcMaxSmem) return -1;
    pcgc_config<T>(s, cs, cfg, at);
    // the rest of the SM's shared/L1 storage stays L1 for the matrix rows
    int dev = 0, smem_sm = 0;
    ZCHECK(cudaGetDevice(&dev));
    ZCHECK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    int pct = (int)std::min<size_t>(100, (100 * (cfg.dynamicSmemBytes + 2048) + smem_sm - 1) / std::max(1, smem_sm));
    ZCHECK(cudaFuncSetAttribute(k_pcg_cluster<T, 1>, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, k_pcg_cluster<T, 1>, &cfg) != cudaSuccess || ncl < 1) {
        cudaGetLastError();
        return -1;
    }
    return cs;
}

// whether cluster size cs can run the cluster solve of this scene
template <class T>
bool pcgc_valid(zema_scene* s, int code) {
    if (sched_binned(code)) {
        const int m = sched_cs(code);
        if ((m != 1 && m != 2 && m != 4) || pcgc_smem<T>(s, code) > (sched_occ(code) == 2 ? kPcgcMaxSmem2 : kPcgcMaxSmem))
            return false;
        const std::vector<int>& off = pcgc_bins(s, m);
        for (int k = 0, cs = 1; k < 5; ++k, cs *= 2) {
            if (off[k + 1] == off[k]) continue;
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            pcgc_config<T>(s, code, cfg, at, cs, off[k + 1] - off[k]);
            int ncl = 0;
            if (cudaOccupancyMaxActiveClusters(&ncl, pcgc_kernel<T>(code), &cfg) != cudaSuccess || ncl < 1) {
                cudaGetLastError();
                return false;
            }
        }
        return true;
    }
    const int cs = sched_cs(code);
    if (cs < 1 || cs > 16 || (s->pcgc_max_soft + cs - 1) / cs > kPcgcOwn * kPcgcThreads ||
        pcgc_smem<T>(s, code) > (sched_occ(code) == 2 ? kPcgcMaxSmem2 : kPcgcMaxSmem))
        return false;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    pcgc_config<T>(s, code, cfg, at);
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, pcgc_kernel<T>(code), &cfg) != cudaSuccess || ncl < 1) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// After a stream synchronisation: the statistics of the solve whose read-back
// was waiting (status, iterations into the step's count, and the solve's
// algorithmic bytes for the live roofline, per iteration the bytes of a
// streaming PCG iteration whose three fused passes keep nothing on chip:
// SpMV, every stored block (9 values + 4 B column) and the row pointers
// (8 B per row), p read, q written; update, x and r read and written, p and
// q read, z written, the preconditioner read (9 values per soft node, 144
// per affine body); direction, z read, p read and written; 36 vector values
// per node in the solve's type).
void pcg_finish(zema_scene* s) {
    if (!s->pcg_pending) return;
    s->pcg_pending = false;
    const int NE = s->n_envs;
    int64_t tot = 0;
    for (int e = 0; e < NE; ++e) {
        if (s->h_pcg[NE + e] == 2) fail(ZEMA_ERR_NONFINITE, "non-finite value in the linear solve");
        if (s->h_pcg[NE + e] == 3)
            fail(ZEMA_ERR_PCG_MAXITER, "linear solve reached max_pcg iterations without meeting its tolerance");
        tot += s->h_pcg[e];
        if (s->pcg_pending_refines) s->S.pcg_refines += s->h_pcg[2 * NE + e];
    }
    s->S.pcg_iters += tot;
    if ((int)s->env_cost.size() == NE)
        for (int e = 0; e < NE; ++e)
            if (s->h_pcg[e] > 0)
                s->env_cost[e] = (double)s->h_pcg[e] * (s->env_node_start_h[e + 1] - s->env_node_start_h[e]);
    if (s->n_cblocks_pending) {  // read back with the solve's statistics
        s->n_cblocks = s->h32[8];
        s->n_cblocks_pending = false;
    }
    const double ts = s->pcg_pending_tsize;
    const double nn = s->n_nodes;
    const double bs = 9.0 * ts + 4.0;  // one stored block and its column index
    const double pre = 9.0 * ts * (nn - 4.0 * s->n_aff) + 144.0 * ts * s->n_aff;
    const double per_it = bs * ((double)s->n_sblocks + (double)s->n_cblocks) + nn * (8.0 + 36.0 * ts) + pre;
    alg_bytes_add(s->pcg_pending_kname, per_it * (double)tot / std::max(1, NE));
}

// ---------------------------------------------------------------------------
// PCG: solve (S + C) p = -g for every env not flagged in done_h (one
// persistent cooperative launch per solve)
// ---------------------------------------------------------------------------
template <class T>
void pcg_t(zema_scene* s, const std::vector<int>& done_h) {
    cudaStream_t st = s->st;
    Geo& G = s->G;
    int NE = s->n_envs;
    Bsr<T> S{s->S_rowptr.p, s->S_col.p, (const T*)s->S_val.p};
    Bsr<T> C{s->C_rowptr.p, s->C_col.p, (const T*)s->C_val.p};
    T* Minv_s = (T*)s->Minv_s.p;
    T* Minv_a = (T*)s->Minv_a.p;
    ZL(k_precond<T>, div_up(s->n_units, 128), 128, 0, st)(G, S, C, Minv_s);
    if (s->n_aff)
        ZL(k_precond_aff<T>, div_up(s->n_aff, kPrecondAffWarps), 32 * kPrecondAffWarps, 0, st)(G, S, C, Minv_a);
    ZL(k_negate, div_up(3 * (size_t)s->n_nodes, TB), TB, 0, st)(s->g.p, s->b.p, 3 * (size_t)s->n_nodes);
    ZLAUNCH();
    for (int e = 0; e < NE; ++e) s->hi[e] = s->hi[3 * NE + e] = done_h[e];
    upload_env_ints(s, s->conv.p, s->hi);
    ZCHECK(cudaMemsetAsync(s->pcg_iters.p, 0, NE * sizeof(int), st));
    const int pi = s->P.precision == 1 ? 1 : 0;
    if (s->P.pcg_kind != 1 && s->pcgc_cs[pi] == 0) {
        if (s->P.pcg_cluster_size > 0) {
            // pinned by the caller
            if (pcgc_choose<T>(s) < 0 || !pcgc_valid<T>(s, s->P.pcg_cluster_size))
                fail(ZEMA_ERR_INVALID_ARG, "pcg_cluster_size cannot run the cluster solve of this scene");
            s->pcgc_cs[pi] = s->P.pcg_cluster_size;
        } else {
            s->pcgc_cs[pi] = pcgc_choose<T>(s);
        }
    }
    if (s->P.pcg_kind == 2 && s->pcgc_cs[pi] < 0)
        fail(ZEMA_ERR_INVALID_ARG, "cluster PCG unavailable for this scene on this device");
    const bool use_cluster = s->P.pcg_kind != 1 && s->pcgc_cs[pi] > 0;
    const char* kname = use_cluster ? "k_pcg_cluster" : "k_pcg_persistent";
    // FP32 cluster solves read the matrix packed (fixed for all solves of
    // this system, refinements included)
    const float4* pk = nullptr;
    if (sizeof(T) == sizeof(float) && use_cluster) {
        s->pk.ensure(&s->A, 3 * ((size_t)s->n_sblocks + s->C_col.cap) + 3);
        ZL(k_pack_blocks, 148 * 8, 256, 0, st)(G, Bsr<float>{S.rowptr, S.col, (const float*)S.val},
                                              Bsr<float>{C.rowptr, C.col, (const float*)C.val}, (int)s->n_sblocks,
                                              s->C_rowptr.p + s->n_nodes, s->pk.p);
        ZLAUNCH();
        pk = s->pk.p;
    }
    // FP32 cluster solves refine against FP64 residuals inside the launch
    // (envs with up to kPcgcRefAff affine bodies), each env on its own as
    // soon as its solve converges; the grid-wide solve refines from the host
    const bool refine_in_launch = sizeof(T) < sizeof(double) && use_cluster && s->pcgc_max_aff <= kPcgcRefAff;
    if (refine_in_launch) s->q.ensure(&s->A, std::max<size_t>(3 * (size_t)s->n_nodes + 3, 3 * (size_t)s->n_sv + 3));
    // the iterations and status of the last launch go to pinned memory, to
    // be read after the next synchronisation (pcg_finish)
    auto collect = [&]() {
        if (s->pcg_pending) {  // never two waiting at once
            ZCHECK(cudaStreamSynchronize(st));
            pcg_finish(s);
        }
        ZCHECK(cudaMemcpyAsync(s->h_pcg, s->pcg_iters.p, NE * sizeof(int), cudaMemcpyDeviceToHost, st));
        ZCHECK(cudaMemcpyAsync(s->h_pcg + NE, s->conv.p, NE * sizeof(int), cudaMemcpyDeviceToHost, st));
        if (refine_in_launch)
            ZCHECK(cudaMemcpyAsync(s->h_pcg + 2 * NE, s->pcg_refines.p, NE * sizeof(int), cudaMemcpyDeviceToHost, st));
        s->pcg_pending_refines = refine_in_launch;
        s->pcg_pending = true;
        s->pcg_pending_tsize = (int)sizeof(T);
        s->pcg_pending_kname = kname;
    };
    // one cluster solve with cs CTAs per env (launch only)
    auto launch_cluster = [&](const double* rhs, double* xo, int cs, const double* tol2_env = nullptr) {
        PcgcArgs<T> c;
        c.G = G;
        c.S = S;
        c.C = C;
        c.b = rhs;
        c.x_out = xo;
        c.z = (T*)s->z.p;
        c.Minv_s = Minv_s;
        c.Minv_a = Minv_a;
        c.conv = s->conv.p;
        c.iters = s->pcg_iters.p;
        c.tol2 = s->P.pcg_rel_tol * s->P.pcg_rel_tol;
        c.tol2_env = tol2_env;
        c.max_iter = s->P.max_pcg;
        c.max_env_nodes = s->pcgc_max_env_nodes;
        c.max_rows = pcgc_max_rows(s, cs);
        c.max_aff = s->pcgc_max_aff;
        c.slice_cap = pcgc_slice_cap<T>(s, cs);
        c.chunk_cap = pcgc_chunk_cap(s, cs);
        c.env_list = nullptr;
        c.pk = pk;
        c.pk_c0 = (int)s->n_sblocks;
        c.refine = refine_in_launch && tol2_env == nullptr ? kPcgcRefine : 0;
        c.r64 = s->q.p;
        c.refines = s->pcg_refines.p;
        if (NE > 1 && !sched_binned(cs)) {
            // launch order by the envs' last solve cost (iterations x nodes;
            // the order changes no env's arithmetic)
            if ((int)s->env_cost.size() != NE) {
                s->env_cost.resize(NE);
                for (int e = 0; e < NE; ++e) s->env_cost[e] = s->env_node_start_h[e + 1] - s->env_node_start_h[e];
            }
            std::vector<int> by_cost(NE), order;
            for (int e = 0; e < NE; ++e) by_cost[e] = e;
            std::stable_sort(by_cost.begin(), by_cost.end(),
                             [&](int a, int b) { return s->env_cost[a] > s->env_cost[b]; });
            // the costliest first, each followed by the cheapest left, so
            // that the clusters resident at once keep a mixed working set
            // (all-large first waves overflow L2 and re-read their matrices
            // from DRAM every iteration)
            order.reserve(NE);
            for (int i = 0, j = NE - 1; i <= j; ++i, --j) {
                order.push_back(by_cost[i]);
                if (i != j) order.push_back(by_cost[j]);
            }
            if (order != s->env_order_h) {
                s->env_order_h = order;
                s->env_order.ensure(&s->A, NE);
                ZCHECK(cudaMemcpyAsync(s->env_order.p, s->env_order_h.data(), NE * sizeof(int),
                                       cudaMemcpyHostToDevice, st));
            }
            c.env_list = s->env_order.p;
        }
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        pcgc_config<T>(s, cs, cfg, at);
        cfg.stream = st;
        if (sched_occ(cs) == 2) {
            // shared memory for two CTAs per SM, the rest L1
            int dev = 0, smem_sm = 0;
            ZCHECK(cudaGetDevice(&dev));
            ZCHECK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
            const int pct = (int)std::min<size_t>(
                100, (100 * 2 * (cfg.dynamicSmemBytes + 8192) + smem_sm - 1) / std::max(1, smem_sm));
            ZCHECK(cudaFuncSetAttribute(k_pcg_cluster<T, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
        }
        if (sched_binned(cs)) {
            // one launch per env group, each with its own cluster size, on
            // streams of their own so that the groups run at once (forked
            // from and joined back into the scene's stream; timed as one)
            const std::vector<int>& off = pcgc_bins(s, sched_cs(cs));
            if (!s->bin_fork) {
                ZCHECK(cudaEventCreateWithFlags(&s->bin_fork, cudaEventDisableTiming));
                for (int k = 0; k < 5; ++k) {
                    ZCHECK(cudaStreamCreateWithFlags(&s->bin_st[k], cudaStreamNonBlocking));
                    ZCHECK(cudaEventCreateWithFlags(&s->bin_join[k], cudaEventDisableTiming));
                }
            }
            LaunchScope region("k_pcg_cluster", false);
            ZCHECK(cudaEventRecord(s->bin_fork, st));
            for (int k = 0, cg = 1; k < 5; ++k, cg *= 2) {
                const int ng = off[k + 1] - off[k];
                if (!ng) continue;
                c.env_list = s->pcgc_bin_list[sched_cs(cs)].p + off[k];
                pcgc_config<T>(s, cs, cfg, at, cg, ng);
                cfg.stream = s->bin_st[k];
                ZCHECK(cudaStreamWaitEvent(s->bin_st[k], s->bin_fork, 0));
                ++launch_counter();
                ZCHECK(cudaLaunchKernelEx(&cfg, pcgc_kernel<T>(cs), c));
                ZCHECK(cudaEventRecord(s->bin_join[k], s->bin_st[k]));
                ZCHECK(cudaStreamWaitEvent(st, s->bin_join[k], 0));
            }
            ZLAUNCH();
            return;
        }
        {
            LaunchScope ls("k_pcg_cluster");
            ZCHECK(cudaLaunchKernelEx(&cfg, pcgc_kernel<T>(cs), c));
        }
        ZLAUNCH();
    };
    // one grid-wide solve (cooperative launch; launch only)
    auto launch_grid = [&](const double* rhs, double* xo, const double* tol2_env) {
        PcgArgs<T> a;
        a.G = G;
        a.S = S;
        a.C = C;
        a.b = rhs;
        a.x_out = xo;
        const size_t nv = 3 * (size_t)s->n_nodes;
        s->pcg_work.ensure(&s->A, 6 * nv);
        T* w = (T*)s->pcg_work.p;
        a.x = w;
        a.r = w + nv;
        a.z = w + 2 * nv;
        a.p = w + 3 * nv;
        a.p2 = w + 4 * nv;
        a.q = w + 5 * nv;
        a.Minv_s = Minv_s;
        a.Minv_a = Minv_a;
        a.T = Tiles{s->n_tiles, s->tile_u0.p, s->tile_u1.p, s->tile_n0.p, s->tile_n1.p, s->tile_env.p, s->env_tile_start.p};
        a.pt_rz = (T*)s->pt_a.p;
        a.pt_rz2 = (T*)s->pt_b.p;
        a.pt_pq = (T*)s->pt_c.p;
        a.pt_rr = (T*)s->pt_d.p;
        a.pt_bb = (T*)s->pt_e.p;
        a.conv = s->conv.p;
        a.iters = s->pcg_iters.p;
        a.tol2 = s->P.pcg_rel_tol * s->P.pcg_rel_tol;
        a.tol2_env = tol2_env;
        a.max_iter = s->P.max_pcg;
        size_t smem = 4 * (size_t)NE * sizeof(double) + 2 * (size_t)NE * sizeof(T) + (size_t)NE * sizeof(int);
        int& grid = s->P.precision == 1 ? s->pcg_grid_f : s->pcg_grid;
        if (grid == 0) {
            int dev = 0, nsm = 0, per = 0;
            ZCHECK(cudaGetDevice(&dev));
            ZCHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
            if (smem > 48 * 1024)
                ZCHECK(cudaFuncSetAttribute(k_pcg_persistent<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            ZCHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_persistent<T>, 256, smem));
            grid = std::max(1, std::min(s->n_tiles, per * nsm));
        }
        void* args[] = {&a};
        {
            LaunchScope ls("k_pcg_persistent");
            ZCHECK(cudaLaunchCooperativeKernel((const void*)k_pcg_persistent<T>, dim3(grid), dim3(256), args, smem, st));
        }
        ZLAUNCH();
    };
    if (use_cluster && s->pcgc_tune[pi]) {
        // autotuner: time the solve of this system with every valid cluster
        // size (results discarded, best of two runs each) and keep the
        // fastest; the solve below then uses it
        s->pcgc_tune[pi] = false;
        s->pcgc_tuned[pi].clear();
        cudaEvent_t e0, e1;
        ZCHECK(cudaEventCreate(&e0));
        ZCHECK(cudaEventCreate(&e1));
        float best = INFINITY;
        int best_cs = s->pcgc_cs[pi];
        for (int code : {1, 2, 4, 8, 16, 101, 102, 104, 108, 116, 1001, 1002, 1004, 1101, 1102, 1104}) {
            const int cs = code;
            if (!pcgc_valid<T>(s, cs)) continue;
            float ms = INFINITY;
            for (int rep = 0; rep < 2; ++rep) {
                upload_env_ints(s, s->conv.p, s->hi + 3 * NE);
                ZCHECK(cudaEventRecord(e0, st));
                launch_cluster(s->b.p, s->r.p, cs);
                ZCHECK(cudaEventRecord(e1, st));
                ZCHECK(cudaEventSynchronize(e1));
                float t = 0.0f;
                ZCHECK(cudaEventElapsedTime(&t, e0, e1));
                ms = std::min(ms, t);
            }
            s->pcgc_tuned[pi].push_back({cs, ms});
            if (ms < best) {
                best = ms;
                best_cs = cs;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        s->pcgc_cs[pi] = best_cs;
        s->pcgc_tuned_flag[pi] = true;
        upload_env_ints(s, s->conv.p, s->hi + 3 * NE);
    }
    if (s->n_sm == 0) {
        int dev = 0;
        ZCHECK(cudaGetDevice(&dev));
        ZCHECK(cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, dev));
    }
    // The tuned schedule is the fastest for the whole batch.  When so few
    // envs still solve that even 16-CTA clusters, one per SM, leave SMs idle
    // (the lockstep tail of the batched Newton loop: one or two stiff envs),
    // the solve is bound by one env's latency instead, and the 16-CTA
    // schedule has the lowest (measured on the single-env grasp: 0.50 ms per
    // solve against 0.92 ms for 8 CTAs two per SM).  Tuned scenes only, so
    // untuned ones stay bit-reproducible.
    auto schedule_for = [&](int n_solving) -> int {
        const int tuned = s->pcgc_cs[pi];
        if (!s->pcgc_tuned_flag[pi] || s->P.pcg_cluster_size > 0 || tuned == 16) return tuned;
        if (n_solving > s->n_sm / 16) return tuned;
        if (s->pcgc_valid16[pi] < 0) s->pcgc_valid16[pi] = pcgc_valid<T>(s, 16) ? 1 : 0;
        return s->pcgc_valid16[pi] ? 16 : tuned;
    };
    // one solve of the selected form, then its statistics
    auto run_solve = [&](const double* rhs, double* xo, const double* tol2_env, int n_solving) {
        // envs skipped by this solve must not count the previous solve's
        // iterations and refinement rounds
        ZCHECK(cudaMemsetAsync(s->pcg_iters.p, 0, NE * sizeof(int), st));
        if (refine_in_launch) ZCHECK(cudaMemsetAsync(s->pcg_refines.p, 0, NE * sizeof(int), st));
        if (use_cluster)
            launch_cluster(rhs, xo, schedule_for(n_solving), tol2_env);
        else
            launch_grid(rhs, xo, tol2_env);
        if (s->fault_armed == ZEMA_FAULT_SOLVE_NONFINITE) {
            ZL(k_fault_solve_status, 1, 128, 0, st)(s->fault_dev.p, s->conv.p, NE);
            ZLAUNCH();
        }
        collect();
    };
    int n_solving = 0;
    for (int e = 0; e < NE; ++e) n_solving += done_h[e] ? 0 : 1;
    run_solve(s->b.p, s->p.p, nullptr, n_solving);
    if (sizeof(T) < sizeof(double) && !refine_in_launch) {
        // FP64 residual refinement of the FP32 solve: r = b - A x with
        // FP64 products; while |r| > tol |b| solve A d = r and add d
        std::vector<int> need(NE);
        for (int e = 0; e < NE; ++e) need[e] = done_h[e] ? 0 : 1;
        const size_t nc = (size_t)NE * kChunks;
        std::vector<double> prr(nc), pbb(nc);
        for (int ref = 0; ref < kPcgcRefine; ++ref) {
            for (int e = 0; e < NE; ++e) s->hi[e] = need[e] ? 0 : 1;
            upload_env_ints(s, s->conv.p, s->hi);
            ZL(k_residual64<T>, div_up(32 * (long long)s->n_nodes, 128), 128, 0, st)(G, S, C, s->p.p, s->b.p,
                                                                                    s->conv.p, s->q.p);
            ZL(k_env_dot2, red_grid(NE), kRedThreads, 0, st)(G, s->b.p, s->q.p, s->part4.p, s->part5.p);
            ZL(k_env_dot2, red_grid(NE), kRedThreads, 0, st)(G, s->q.p, s->b.p, s->part6.p, s->part7.p);
            ZLAUNCH();
            ZCHECK(cudaMemcpyAsync(prr.data(), s->part5.p, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
            ZCHECK(cudaMemcpyAsync(pbb.data(), s->part7.p, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
            ZCHECK(cudaStreamSynchronize(st));
            pcg_finish(s);  // the solve before this residual
            int count = 0;
            const double tol2 = s->P.pcg_rel_tol * s->P.pcg_rel_tol;
            for (int e = 0; e < NE; ++e) {
                s->hd[e] = tol2;
                if (!need[e]) continue;
                double rr = 0.0, bbv = 0.0;
                for (int k = 0; k < kChunks; ++k) {
                    rr += prr[(size_t)e * kChunks + k];
                    bbv += pbb[(size_t)e * kChunks + k];
                }
                if (!std::isfinite(rr)) fail(ZEMA_ERR_NONFINITE, "non-finite residual of the linear solve");
                need[e] = rr > tol2 * bbv ? 1 : 0;
                count += need[e];
                // the correction d only has to bring |r - A d| under
                // tol |b|: stop its solve at half of that, relative to |r|
                if (need[e]) s->hd[e] = std::min(0.25, 0.25 * tol2 * bbv / rr);
            }
            if (!count) break;
            s->S.pcg_refines += count;
            for (int e = 0; e < NE; ++e) s->hi[e] = need[e] ? 0 : 1;
            upload_env_ints(s, s->conv.p, s->hi);
            upload_env_doubles(s, s->tol2_env.p, s->hd);
            run_solve(s->q.p, s->r.p, s->tol2_env.p, count);
            for (int e = 0; e < NE; ++e) s->hi[e] = need[e];
            upload_env_ints(s, s->need.p, s->hi);
            ZL(k_add_env, div_up(s->n_nodes, TB), TB, 0, st)(G, s->p.p, s->r.p, s->need.p);
            ZLAUNCH();
        }
    }
    // done envs: zero direction
    for (int e = 0; e < NE; ++e) s->hi[e] = done_h[e];
    upload_env_ints(s, s->need.p, s->hi);
    ZL(k_mask_env, div_up(s->n_nodes, TB), TB, 0, st)(G, s->p.p, s->need.p);
    ZLAUNCH();
}

// The solve of the Newton system; its statistics and status are read back
// with the step-norm test (pcg_finish after step_norm).
void pcg(zema_scene* s, const std::vector<int>& done_h) {
    if (s->P.precision == 1)
        pcg_t<float>(s, done_h);
    else
        pcg_t<double>(s, done_h);
}

// per-env max step component -> s->hd
void step_norm(zema_scene* s) {
    cudaStream_t st = s->st;
    int NE = s->n_envs;
    ZL(k_step_norm, red_grid(NE), kRedThreads, 0, st)(s->G, s->p.p, s->part7.p);
    ZL(k_max_total, div_up(NE, 64), 64, 0, st)(s->part7.p, NE, s->E.p);
    ZLAUNCH();
    const bool probe = s->fault_armed == ZEMA_FAULT_STATUS;
    if (probe) {
        ZL(k_fault_status_word, 1, 32, 0, st)(s->fault_dev.p);
        ZLAUNCH();
        ZCHECK(cudaMemcpyAsync(s->hi, s->fault_dev.p + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    ZCHECK(cudaMemcpyAsync(s->hd, s->E.p, NE * sizeof(double), cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaStreamSynchronize(st));
    if (probe && s->hi[0] != 0) fail(s->hi[0], "fault injected by zema_inject_fault");
}

// Swept candidates of the motion from x along dir (alpha = 1): X = X(x), q =
// X(x + dir) (kept in q, which energy() does not overwrite), the pairs into
// s->swept / s->swept_env and their count into s->n_swept; converged envs
// (done_h) take no step and stay out; s->alpha is left at 1 for every env.
void swept_candidates(zema_scene* s, const double* dir, const std::vector<int>& done_h) {
    cudaStream_t st = s->st;
    Geo& G = s->G;
    int NE = s->n_envs;
    ZL(k_sv_pos, div_up(s->n_sv, TB), TB, 0, st)(G, s->x.p, s->X.p);
    std::vector<double> one(NE, 1.0);
    ZCHECK(cudaMemcpyAsync(s->alpha.p, one.data(), NE * sizeof(double), cudaMemcpyHostToDevice, st));
    ZL(k_axpy_env, div_up(s->n_nodes, TB), TB, 0, st)(G, s->x.p, dir, s->alpha.p, s->xtrial.p);
    ZL(k_sv_pos, div_up(s->n_sv, TB), TB, 0, st)(G, s->xtrial.p, s->X1.p);
    ZLAUNCH();
    // X1 is overwritten by energy(); keep the swept end positions in q (scratch)
    s->q.ensure(&s->A, std::max<size_t>(3 * (size_t)s->n_nodes + 3, 3 * (size_t)s->n_sv + 3));
    ZCHECK(cudaMemcpyAsync(s->q.p, s->X1.p, 3 * (size_t)s->n_sv * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // converged envs take no step: their primitives stay out of the swept
    // broad phase and the ACCD
    bool any_done = false;
    for (int e = 0; e < NE; ++e) any_done |= done_h[e] != 0;
    if (any_done) {
        for (int e = 0; e < NE; ++e) s->hi[e] = done_h[e] ? 1 : 0;
        upload_env_ints(s, s->skip.p, s->hi);
    }
    int e_lo = 0, e_hi = NE - 1;
    active_range(done_h, e_lo, e_hi);
    s->n_swept = candidates(s, s->X.p, s->q.p, s->swept, s->swept_env, any_done ? s->skip.p : nullptr, e_lo, e_hi);
}

// Line search along direction dir from x (Newton step or warm-start
// proposal): ACCD bound over the swept candidates, then halving until
// E(x + alpha dir) <= E(x) per env.  On success x is advanced.  Returns the
// number of halvings, or -1 when an env fails.
//
// e_at_x (nullable, per env): in, the potential at x where known (NaN where
// not); out, the potential at the new x.  The potential at x does not depend
// on which swept list its barrier is summed over, as long as the list holds
// every pair with d < dhat at x, and every list built from a motion that
// starts at x does; so an env's value from the line search that reached x
// stands in for a new evaluation (only the order of the sum differs).
int line_search(zema_scene* s, const double* dir, const std::vector<int>& done_h, bool warm,
                std::vector<int>* accepted, int warm_halvings = 0, bool strict = false,
                std::vector<double>* e_at_x = nullptr, bool swept_ready = false) {
    // warm-start proposals get warm_halvings halvings (default: a single energy
    // check), Newton steps up to 60; strict: a step must lower the energy
    // (the learned correction), otherwise it may also keep it equal
    const int max_halvings = warm ? warm_halvings : 60;
    cudaStream_t st = s->st;
    Geo& G = s->G;
    int NE = s->n_envs;
    double t0 = now_ms();
    // swept candidates X(x) -> X(x + dir) (unless the step's start built them
    // for this direction already); alpha = 1 on the device
    uint32_t ns;
    if (swept_ready) {
        std::vector<double> one(NE, 1.0);
        ZCHECK(cudaMemcpyAsync(s->alpha.p, one.data(), NE * sizeof(double), cudaMemcpyHostToDevice, st));
        ns = s->n_swept;
    } else {
        swept_candidates(s, dir, done_h);
        ns = s->n_swept;
    }
    ZCHECK(cudaMemsetAsync(s->capflag.p, 0, sizeof(int), st));
    if (ns) ZL(k_accd, div_up(ns, 128), 128, 0, st)(G, s->X.p, s->q.p, s->swept.p, (int)ns, s->alpha.p, s->capflag.p);
    ZLAUNCH();
    // the first trial takes the ACCD bounds where they are, on the device; the
    // host reads them back with that trial's energies (no round trip here)
    std::vector<double> alpha(NE);
    ZCHECK(cudaMemcpyAsync(s->h_alpha, s->alpha.p, NE * sizeof(double), cudaMemcpyDeviceToHost, st));
    bool alpha_known = false;
    s->S.ms_phase[4] += now_ms() - t0;
    t0 = now_ms();
    bool need_e0 = e_at_x == nullptr;
    if (e_at_x)
        for (int e = 0; e < NE; ++e) need_e0 |= !done_h[e] && std::isnan((*e_at_x)[e]);
    std::vector<double> E0(NE, 0.0);
    if (need_e0 && e_at_x) {
        // only the envs whose potential at x is not known evaluate it
        const int* const keep_mask = G.env_done;
        for (int e = 0; e < NE; ++e) s->hi[e] = done_h[e] || !std::isnan((*e_at_x)[e]) ? 1 : 0;
        upload_env_ints(s, s->ls_skip.p, s->hi);
        G.env_done = s->ls_skip.p;
        energy(s, s->x.p, s->swept.p, s->swept_env.p);
        G.env_done = keep_mask;
        for (int e = 0; e < NE; ++e) E0[e] = std::isnan((*e_at_x)[e]) ? s->hd[e] : (*e_at_x)[e];
    } else if (need_e0) {
        energy(s, s->x.p, s->swept.p, s->swept_env.p);
        E0.assign(s->hd, s->hd + NE);
    } else {
        E0 = *e_at_x;
    }
    std::vector<double> Eacc(E0);  // the potential at the accepted point, per env
    std::vector<int> acc(NE, 0);
    for (int e = 0; e < NE; ++e)
        if (done_h[e]) acc[e] = 1;  // converged: no step (its direction is zero)
    int halvings = 0;
    bool fail_ls = false;
    // after the first trial only the envs still halving evaluate the
    // potential: the others (converged, or accepted already) are masked for
    // the energy kernels, whose per-env sums do not depend on one another
    const int* const done_mask = G.env_done;
    struct RestoreMask {
        Geo& G;
        const int* m;
        ~RestoreMask() { G.env_done = m; }
    } restore_mask{G, done_mask};
    for (int k = 0; k <= max_halvings; ++k) {
        if (alpha_known)
            ZCHECK(cudaMemcpyAsync(s->alpha.p, alpha.data(), NE * sizeof(double), cudaMemcpyHostToDevice, st));
        ZL(k_axpy_env, div_up(s->n_nodes, TB), TB, 0, st)(G, s->x.p, dir, s->alpha.p, s->xtrial.p);
        ZLAUNCH();
        if (k > 0) {
            for (int e = 0; e < NE; ++e) s->hi[e] = acc[e] ? 1 : 0;
            upload_env_ints(s, s->ls_skip.p, s->hi);
            G.env_done = s->ls_skip.p;
        }
        energy(s, s->xtrial.p, s->swept.p, s->swept_env.p);
        if (!alpha_known) {
            alpha.assign(s->h_alpha, s->h_alpha + NE);
            for (int e = 0; e < NE; ++e)
                if (done_h[e]) alpha[e] = 0.0;
            alpha_known = true;
        }
        if (!warm && s->fault_armed == ZEMA_FAULT_NO_DECREASE)
            for (int e = 0; e < NE; ++e) s->hd[e] = INFINITY;  // every trial point rejected
        bool all = true;
        for (int e = 0; e < NE; ++e) {
            if (acc[e]) continue;
            if (strict ? s->hd[e] < E0[e] : s->hd[e] <= E0[e]) {
                acc[e] = 1;
                Eacc[e] = s->hd[e];
            } else if (k < max_halvings) {
                alpha[e] *= 0.5;
                ++halvings;
                all = false;
            } else {
                all = false;
            }
        }
        if (all) break;
        if (k == max_halvings) fail_ls = true;
    }
    if (fail_ls && !warm) {
        s->S.ms_phase[1] += now_ms() - t0;
        return -1;
    }
    // envs that never accepted (warm start only): alpha = 0
    for (int e = 0; e < NE; ++e)
        if (!acc[e]) {
            alpha[e] = 0.0;
            Eacc[e] = E0[e];
        }
    if (accepted) *accepted = acc;
    if (e_at_x) *e_at_x = Eacc;
    ZCHECK(cudaMemcpyAsync(s->alpha.p, alpha.data(), NE * sizeof(double), cudaMemcpyHostToDevice, st));
    ZL(k_axpy_env, div_up(s->n_nodes, TB), TB, 0, st)(G, s->x.p, dir, s->alpha.p, s->xtrial.p);
    ZLAUNCH();
    ZCHECK(cudaMemcpyAsync(s->x.p, s->xtrial.p, 3 * (size_t)s->n_nodes * sizeof(double), cudaMemcpyDeviceToDevice, st));
    s->S.ms_phase[1] += now_ms() - t0;
    return halvings;
}

// lag friction at the current x (= x^t): records, weights, normals, mu lambda
// (list: a candidate list that holds every pair with d < dhat at x, such as
// the swept candidates of a motion starting at x; NULL: a broad phase at x)
void lag_friction(zema_scene* s, const PairRec* list = nullptr, const uint32_t* list_env = nullptr,
                  uint32_t n_list = 0) {
    cudaStream_t st = s->st;
    ZL(k_sv_pos, div_up(s->n_sv, TB), TB, 0, st)(s->G, s->x.p, s->Xt.p);
    ZLAUNCH();
    uint32_t na = list ? active_from(s, s->Xt.p, list, list_env, n_list, false) : active_pairs(s, s->Xt.p, false);
    s->lag.ensure(&s->A, na + 1);
    s->lag_w.ensure(&s->A, 4 * (size_t)na + 4);
    s->lag_n.ensure(&s->A, 3 * (size_t)na + 3);
    s->lag_c.ensure(&s->A, na + 1);
    if (na) {
        ZCHECK(cudaMemcpyAsync(s->lag.p, s->act.p, na * sizeof(PairRec), cudaMemcpyDeviceToDevice, st));
        ZL(k_lag_friction, div_up(na, 128), 128, 0, st)(s->G, s->Xt.p, s->lag.p, (int)na, s->kappa.p, s->lag_w.p,
                                                         s->lag_n.p, s->lag_c.p);
        ZLAUNCH();
    }
    ZCHECK(cudaMemcpyAsync(s->lag_env.p, s->act_env.p, (s->n_envs + 1) * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    s->n_lag = na;
}

// kappa: kappa_min = 1e3 x mean soft lumped mass of the env (else mean
// dynamic affine mass / 8); kappa = clamp(-gE . gB / |gB|^2, kappa_min,
// 100 kappa_min) at x^t with gE the gradient without contact terms and gB the
// barrier gradient for kappa = 1, both in the paper's DOF coordinates.
void init_kappa(zema_scene* s) {
    cudaStream_t st = s->st;
    int NE = s->n_envs;
    bool any = false;
    for (int e = 0; e < NE; ++e) any |= !s->kappa_ready[e];
    if (!any) return;
    std::vector<double> kmin(NE, 1.0);
    for (int e = 0; e < NE; ++e) {
        double sm = 0.0;
        int cnt = 0;
        for (int n = s->env_node_start_h[e]; n < s->env_node_start_h[e + 1]; ++n)
            if (s->node_mass_h[n] > 0.0) {
                sm += s->node_mass_h[n];
                ++cnt;
            }
        double mbar = 1.0;
        if (cnt) {
            mbar = sm / cnt;
        } else {
            double tot = 0.0;
            int cc = 0;
            for (size_t i = 0; i < s->ain.size(); ++i)
                if (s->ain[i].env == e && s->ain[i].mode == 0) {
                    tot += s->aff_m_in[i] / 8.0;
                    ++cc;
                }
            if (cc) mbar = tot / cc;
        }
        kmin[e] = 1e3 * mbar;
    }
    std::vector<double> kap_cur(NE), kmin_cur(NE);
    ZCHECK(cudaMemcpyAsync(kap_cur.data(), s->kappa.p, NE * sizeof(double), cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaMemcpyAsync(kmin_cur.data(), s->kappa_min.p, NE * sizeof(double), cudaMemcpyDeviceToHost, st));
    std::vector<double> one(NE, 1.0);
    ZCHECK(cudaMemcpyAsync(s->kappa.p, one.data(), NE * sizeof(double), cudaMemcpyHostToDevice, st));
    ZL(k_sv_pos, div_up(s->n_sv, TB), TB, 0, st)(s->G, s->x.p, s->X.p);
    ZLAUNCH();
    active_pairs(s, s->X.p, false);
    uint32_t keep_lag = s->n_lag;
    s->n_lag = 0;
    size_t n3 = 3 * (size_t)s->n_nodes;
    grad_hess(s, false, false, false);
    ZL(k_affine_grad_to_row, div_up(s->n_aff + 1, 64), 64, 0, st)(s->G, s->g.p);
    ZCHECK(cudaMemcpyAsync(s->r.p, s->g.p, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    grad_hess(s, true, false, false);
    ZL(k_affine_grad_to_row, div_up(s->n_aff + 1, 64), 64, 0, st)(s->G, s->g.p);
    ZLAUNCH();
    s->n_lag = keep_lag;
    std::vector<double> ga(n3), ge(n3);
    ZCHECK(cudaMemcpyAsync(ga.data(), s->g.p, n3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaMemcpyAsync(ge.data(), s->r.p, n3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaStreamSynchronize(st));
    for (size_t i = 0; i < n3; ++i) ga[i] -= ge[i];
    ZCHECK(cudaMemcpyAsync(s->z.p, ga.data(), n3 * sizeof(double), cudaMemcpyHostToDevice, st));
    ZL(k_env_dot2, red_grid(NE), kRedThreads, 0, st)(s->G, s->r.p, s->z.p, s->part2.p, s->part3.p);
    ZLAUNCH();
    std::vector<double> pab((size_t)NE * kChunks), pbb((size_t)NE * kChunks);
    ZCHECK(cudaMemcpyAsync(pab.data(), s->part2.p, pab.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaMemcpyAsync(pbb.data(), s->part3.p, pbb.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaStreamSynchronize(st));
    for (int e = 0; e < NE; ++e) {
        if (s->kappa_ready[e]) continue;
        double ab = 0.0, bbv = 0.0;
        for (int c = 0; c < kChunks; ++c) {
            ab += pab[(size_t)e * kChunks + c];
            bbv += pbb[(size_t)e * kChunks + c];
        }
        double k = kmin[e];
        if (bbv > 0.0) k = std::min(std::max(-ab / bbv, kmin[e]), 100.0 * kmin[e]);
        kap_cur[e] = k;
        kmin_cur[e] = kmin[e];
        s->kappa_ready[e] = 1;
    }
    ZCHECK(cudaMemcpyAsync(s->kappa.p, kap_cur.data(), NE * sizeof(double), cudaMemcpyHostToDevice, st));
    ZCHECK(cudaMemcpyAsync(s->kappa_min.p, kmin_cur.data(), NE * sizeof(double), cudaMemcpyHostToDevice, st));
    ZCHECK(cudaStreamSynchronize(st));
}

}  // namespace

namespace {

__global__ void k_scale_dir(Geo G, const double* v, double h, double* d) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.n_nodes) return;
    for (int j = 0; j < 3; ++j) d[3 * (size_t)n + j] = G.node_fixed[n] ? 0.0 : h * v[3 * (size_t)n + j];
}

// free-fall displacement of one step, the scale of the warm-start network's
// displacement features and outputs
double ws_scale(const zema_scene* s) {
    const double* g = s->P.gravity;
    const double gn = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    return s->P.dt * s->P.dt * (gn > 0.0 ? gn : 9.81);
}

// warm-start features at x^t of the soft vertices into s->ws_feat and of the
// dynamic affine bodies into s->ws_afeat (needs the predictor and the lagged
// pairs of this step)
void ws_features(zema_scene* s) {
    cudaStream_t st = s->st;
    if (!s->ws_ns && !s->ws_na) return;
    ZCHECK(cudaMemsetAsync(s->ws_best.p, 0xFF, (size_t)s->n_nodes * sizeof(unsigned long long), st));
    if (s->n_lag)
        ZL(k_ws_nearest, div_up(s->n_lag, 128), 128, 0, st)(s->G, s->Xt.p, s->lag.p, s->lag_w.p, (int)s->n_lag,
                                                           s->ws_best.p);
    if (s->ws_ns) {
        ZL(k_ws_centroid, s->ws_nb, kRedThreads, 0, st)(s->x.p, s->tb_node0.p, s->tb_nv.p, s->tb_c.p);
        ZL(k_ws_features, div_up(s->ws_ns, 128), 128, 0, st)(s->G, s->ws_soft.p, s->ws_body.p, s->ws_ns, s->x.p,
                                                            s->v.p, s->xhat.p, s->tb_c.p, s->tb_R.p, s->ws_best.p,
                                                            s->lag.p, s->lag_w.p, s->lag_n.p, s->P.dt, ws_scale(s),
                                                            s->ws_feat.p);
    }
    if (s->ws_na)
        ZL(k_ws_aff_features, div_up(s->ws_na, 64), 64, 0, st)(s->G, s->ws_aff.p, s->ws_na, s->x.p, s->v.p,
                                                              s->xhat.p, s->ws_aR.p, s->ws_envc.p, s->ws_envd.p,
                                                              s->ws_best.p, s->lag.p, s->lag_w.p, s->lag_n.p,
                                                              s->P.dt, ws_scale(s), s->ws_afeat.p);
    ZLAUNCH();
}

void restore_step(zema_scene* s, bool all = true);

// One time step of every environment.
// lambda_A <- 2 lambda_A - lambda_prev, lambda_prev <- the old lambda_A, for
// the kinematic bodies (the others keep lambda_A = 0)
__global__ void k_al_extrapolate(Geo G, double* lamA, double* lam_prev) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 12 * G.n_aff || G.aff_mode[i / 12] != 2) return;
    const double l = lamA[i];
    lamA[i] = 2.0 * l - lam_prev[i];
    lam_prev[i] = l;
}

void do_step(zema_scene* s) {
    zema_scene& W = *s;
    cudaStream_t st = s->st;
    Geo& G = s->G;
    int NE = s->n_envs;
    size_t n3 = 3 * (size_t)s->n_nodes;
    double t0 = now_ms();
    W.kap_save.ensure(&s->A, 2 * (size_t)NE);
    ZCHECK(cudaMemcpyAsync(W.kap_save.p, s->kappa.p, NE * sizeof(double), cudaMemcpyDeviceToDevice, st));
    ZCHECK(cudaMemcpyAsync(W.kap_save.p + NE, s->kappa_min.p, NE * sizeof(double), cudaMemcpyDeviceToDevice, st));
    W.kappa_ready_save = s->kappa_ready;
    W.dmin_last_save = W.dmin_last;
    W.first_step_done_save = s->first_step_done;
    W.lam_save.ensure(&s->A, 12 * (size_t)s->n_aff + 12);
    if (s->n_aff && s->P.al_extrapolate) {
        // the multipliers start at the extrapolation of the last two steps';
        // the values before it are kept for a full restore
        const size_t na12 = 12 * (size_t)s->n_aff;
        W.lam_hist.ensure(&s->A, 2 * na12 + 12);
        ZCHECK(cudaMemcpyAsync(W.lam_hist.p, s->lamA.p, na12 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        ZCHECK(cudaMemcpyAsync(W.lam_hist.p + na12, s->lamA_prev.p, na12 * sizeof(double), cudaMemcpyDeviceToDevice,
                               st));
        ZL(k_al_extrapolate, div_up(na12, 128), 128, 0, st)(G, s->lamA.p, s->lamA_prev.p);
        ZLAUNCH();
    }
    if (s->n_aff)
        ZCHECK(cudaMemcpyAsync(W.lam_save.p, s->lamA.p, 12 * (size_t)s->n_aff * sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
    if (G.n_joints)
        ZCHECK(cudaMemcpyAsync(W.lamJ_save.p, s->lamJ.p, 12 * (size_t)G.n_joints * sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
    // predictor (Eq. 1-3)
    const double* gr = s->P.gravity;
    ZL(k_predict, div_up(s->n_nodes, TB), TB, 0, st)(G, s->x.p, s->v.p, s->xt.p, s->xhat.p, gr[0], gr[1], gr[2]);
    if (s->n_aff) ZL(k_predict_affine, div_up(s->n_aff, 64), 64, 0, st)(G, s->xhat.p, gr[0], gr[1], gr[2]);
    ZLAUNCH();
    bool first = !s->first_step_done;
    init_kappa(s);
    // the constant-velocity warm start's swept candidates (x^t -> x^t + h v)
    // hold every pair with d < dhat at x^t: one broad phase serves both the
    // friction lagging and the warm start's line search
    W.dirw.ensure(&s->A, n3 + 3);
    ZL(k_scale_dir, div_up(s->n_nodes, TB), TB, 0, st)(G, s->v.p, s->P.dt, W.dirw.p);
    ZLAUNCH();
    swept_candidates(s, W.dirw.p, std::vector<int>(NE, 0));
    bool swept_fresh = true;
    // lagged friction at x^t (Eq. 9-10); d_min at x^t for the kappa rule
    lag_friction(s, s->swept.p, s->swept_env.p, s->n_swept);
    if (first) {
        // d_min over active pairs at x^t
        ZL(k_sv_pos, div_up(s->n_sv, TB), TB, 0, st)(G, s->x.p, s->X.p);
        ZLAUNCH();
        active_pairs(s, s->X.p, true);
        W.dmin_last.assign(NE, INFINITY);
        ZCHECK(cudaMemcpyAsync(s->hd, s->dmin.p, NE * sizeof(double), cudaMemcpyDeviceToHost, st));
        ZCHECK(cudaStreamSynchronize(st));
        for (int e = 0; e < NE; ++e) W.dmin_last[e] = s->hd[e];
        s->first_step_done = true;
    }
    s->S.ms_phase[0] += now_ms() - t0;
    // warm start: x^t + alpha h v^t, CCD-bounded, kept if the energy does not
    // rise; with the learned network, its predicted correction s y is then
    // applied the same way from there (CCD-bounded, kept only if it lowers the
    // energy further), so the learned start is never worse in energy than
    // the constant-velocity one
    W.dirw.ensure(&s->A, n3 + 3);
    const bool learned_soft = s->P.warm_start == 1 && s->ws_net && s->ws_ns;
    const bool learned_aff = s->P.warm_start == 1 && s->ws_anet && s->ws_na;
    const bool learned = learned_soft || learned_aff;
    if (learned || s->rec_feat || s->rec_afeat) ws_features(s);
    if (s->rec_feat && s->ws_ns)
        ZCHECK(cudaMemcpyAsync(s->rec_feat, s->ws_feat.p, (size_t)kWsFeatures * s->ws_ns * sizeof(float),
                               cudaMemcpyDeviceToDevice, st));
    if (s->rec_afeat && s->ws_na)
        ZCHECK(cudaMemcpyAsync(s->rec_afeat, s->ws_afeat.p, (size_t)kWsAffFeatures * s->ws_na * sizeof(float),
                               cudaMemcpyDeviceToDevice, st));
    if (learned_soft) s->ws_net->forward(s->ws_feat.p, s->ws_ns, s->ws_out.p);
    if (learned_aff) s->ws_anet->forward(s->ws_afeat.p, s->ws_na, s->ws_aout.p);
    // one attempt at the step from x^t: warm start, then Newton with the
    // kinematic augmented-Lagrangian rounds; returns the AL rounds
    auto solve = [&](bool use_learned) -> int {
        ZL(k_scale_dir, div_up(s->n_nodes, TB), TB, 0, st)(G, s->v.p, s->P.dt, W.dirw.p);
        ZLAUNCH();
        std::vector<int> done(NE, 0), acc;
        std::vector<double> e_at_x(NE, NAN);  // the potential at the current x, per env
        line_search(s, W.dirw.p, done, true, &acc, 0, false, &e_at_x, swept_fresh);
        swept_fresh = false;  // later line searches overwrite the list
        if (use_learned) {
            ZCHECK(cudaMemsetAsync(W.dirw.p, 0, n3 * sizeof(double), st));
            if (learned_soft)
                ZL(k_ws_direction, div_up(s->ws_ns, 128), 128, 0, st)(s->ws_soft.p, s->ws_ns, s->ws_out.p,
                                                                     ws_scale(s), W.dirw.p);
            if (learned_aff)
                ZL(k_ws_aff_direction, div_up(s->ws_na, 64), 64, 0, st)(G, s->ws_aff.p, s->ws_na, s->ws_aR.p,
                                                                       s->ws_aout.p, ws_scale(s), W.dirw.p);
            ZLAUNCH();
            std::vector<int> acc2;
            line_search(s, W.dirw.p, done, true, &acc2, kWsHalvings, true, &e_at_x);
            for (int e = 0; e < NE; ++e) s->S.warm_learned += acc2[e];
        }
        for (int e = 0; e < NE; ++e) s->S.warm_accepted += acc[e];
        int rounds = 0;
        // while Newton runs, the per-iteration kernels skip converged envs
        // (flagged in s->skip, kept equal to `done`); off again on every exit
        struct DoneMask {
            Geo& G;
            ~DoneMask() { G.env_done = nullptr; }
        } done_mask{G};
        // Newton with the kinematic augmented-Lagrangian rounds of Eq. 13 per
        // env: when an env's step falls under the tolerance, its constraint
        // is checked at that x (read back with the step norm); an env that
        // needs a round gets its multipliers updated and goes on iterating at
        // once, with a zero step in that iteration's line search (so its pairs
        // at x enter the next swept list), instead of waiting for the whole
        // batch to converge and restarting then.  An env's arithmetic is the
        // same either way.  Each round restarts the env's Newton count.
        std::vector<int> env_rounds(NE, 0), env_it(NE, 0), resume(NE, 0);
        int* need_h = s->hi + 2 * NE;  // pinned: the AL check, read back with the step norm
        const bool al = s->n_aff > 0;
        bool converged = false;
        for (;;) {
            bool over = false;
            for (int e = 0; e < NE; ++e)
                if (!done[e]) {
                    over |= env_it[e] >= s->P.max_newton;
                    ++env_it[e];
                }
            if (over) break;
            double ta = now_ms();
            ZL(k_sv_pos, div_up(s->n_sv, TB), TB, 0, st)(G, s->x.p, s->X.p);
            ZLAUNCH();
            // x was reached by a line search along the last swept motion (the
            // warm start or the previous Newton step, a zero one for an env
            // resuming after an AL round), so that swept candidate list
            // contains every pair with d < dhat at x
            for (int e = 0; e < NE; ++e) s->hi[e] = done[e] ? 1 : 0;
            upload_env_ints(s, s->skip.p, s->hi);
            G.env_done = s->skip.p;
            active_from(s, s->X.p, s->swept.p, s->swept_env.p, s->n_swept, true, s->skip.p);
            double tb = now_ms();
            s->S.ms_phase[0] += tb - ta;
            grad_hess(s);  // no read-back: the solve's is the next
            // fault injection: armed for this iteration only (one shot)
            s->fault_armed = 0;
            if (s->fault_kind && s->newton_count == s->fault_at) {
                s->fault_armed = s->fault_kind;
                s->fault_kind = 0;
                const int on[2] = {1, 0};
                ZCHECK(cudaMemcpyAsync(s->fault_dev.p, on, 2 * sizeof(int), cudaMemcpyHostToDevice, st));
            }
            ++s->newton_count;
            double tc = now_ms();
            s->S.ms_phase[2] += tc - tb;
            pcg(s, done);
            if (al) {
                ZCHECK(cudaMemsetAsync(s->need.p, 0, NE * sizeof(int), st));
                ZL(k_al_check, div_up(s->n_aff, 64), 64, 0, st)(G, s->x.p, kin(s), s->tolv.p, s->need.p);
                if (G.n_joints)
                    ZL(k_joint_check, div_up(G.n_joints, 64), 64, 0, st)(G, s->x.p, s->tolv.p,
                                                                        s->P.newton_tol_rel, s->need.p);
                ZLAUNCH();
                ZCHECK(cudaMemcpyAsync(need_h, s->need.p, NE * sizeof(int), cudaMemcpyDeviceToHost, st));
            }
            step_norm(s);
            pcg_finish(s);  // the solve's status and statistics, read back with the step norm
            s->S.ms_phase[3] += now_ms() - tc;
            bool all = true, any_resume = false;
            for (int e = 0; e < NE; ++e) {
                resume[e] = 0;
                if (done[e]) continue;
                if (s->hd[e] <= s->tol_h[e]) {
                    if (al && need_h[e] && env_rounds[e] < s->P.max_al_rounds) {
                        resume[e] = 1;
                        ++env_rounds[e];
                        env_it[e] = 0;
                        e_at_x[e] = NAN;  // the multipliers change the potential
                        any_resume = true;
                        all = false;
                    } else {
                        done[e] = 1;
                    }
                } else {
                    all = false;
                    s->S.newton_iters += 1;
                }
            }
            if (any_resume) {
                upload_env_ints(s, s->need.p, resume.data());
                ZL(k_al_update, div_up(s->n_aff, 64), 64, 0, st)(G, s->x.p, s->qtarget.p, s->lamA.p, s->need.p);
                if (G.n_joints)
                    ZL(k_joint_update, div_up(G.n_joints, 64), 64, 0, st)(G, s->x.p, s->lamJ.p, s->need.p);
                ZLAUNCH();
            }
            if (all) {
                converged = true;
                break;
            }
            // zero the direction of envs that just converged or resume
            for (int e = 0; e < NE; ++e) s->hi[e] = done[e] || resume[e] ? 1 : 0;
            upload_env_ints(s, s->need.p, s->hi);
            ZL(k_mask_env, div_up(s->n_nodes, TB), TB, 0, st)(G, s->p.p, s->need.p);
            ZLAUNCH();
            int hv = line_search(s, s->p.p, done, false, nullptr, 0, false, &e_at_x);
            if (hv < 0) fail(ZEMA_ERR_LINESEARCH, "line search found no decrease after 60 halvings");
            s->S.ls_halvings += hv;
        }
        G.env_done = nullptr;
        if (!converged) fail(ZEMA_ERR_NEWTON_MAXITER, "Newton did not converge within max_newton iterations");
        for (int e = 0; e < NE; ++e) rounds = std::max(rounds, env_rounds[e]);
        return rounds;
    };
    int rounds = 0;
    if (learned) {
        try {
            rounds = solve(true);
        } catch (const ZemaError& e) {
            if (e.status != ZEMA_ERR_NEWTON_MAXITER && e.status != ZEMA_ERR_LINESEARCH) throw;
            // the learned start did not converge: plain Newton from the
            // constant-velocity start decides the step
            restore_step(s, false);  // the step's kappa stays
            s->S.warm_fallback += 1;
            rounds = solve(false);
        }
    } else {
        rounds = solve(false);
    }
    s->S.al_rounds += rounds;
    // with the extrapolation, one more multiplier update from the accepted
    // state (no new solve), so that the values the next step extrapolates
    // from carry no part of the deviation the tolerance let through
    if (s->n_aff && s->P.al_extrapolate) {
        ZL(k_al_update, div_up(s->n_aff, 64), 64, 0, st)(G, s->x.p, s->qtarget.p, s->lamA.p, nullptr);
        ZLAUNCH();
    }
    // d_min at the accepted state (last active-pair pass) and energy of env 0
    std::vector<double> dm(NE);
    ZCHECK(cudaMemcpyAsync(dm.data(), s->dmin.p, NE * sizeof(double), cudaMemcpyDeviceToHost, st));
    // velocities (Eq. 11)
    ZL(k_velocity, div_up(s->n_nodes, TB), TB, 0, st)(G, s->x.p, s->xt.p, s->v.p);
    ZLAUNCH();
    if (s->rec_targ && s->ws_ns) {
        ZL(k_ws_target, div_up(s->ws_ns, 128), 128, 0, st)(s->ws_soft.p, s->ws_ns, s->x.p, s->xt.p, s->ws_feat.p,
                                                          ws_scale(s), s->rec_targ);
        ZLAUNCH();
    }
    if (s->rec_atarg && s->ws_na) {
        ZL(k_ws_aff_target, div_up(s->ws_na, 64), 64, 0, st)(G, s->ws_aff.p, s->ws_na, s->ws_aR.p, s->x.p, s->xt.p,
                                                            s->ws_afeat.p, ws_scale(s), s->rec_atarg);
        ZLAUNCH();
    }
    std::vector<double> kap(NE), kmin(NE);
    ZCHECK(cudaMemcpyAsync(kap.data(), s->kappa.p, NE * sizeof(double), cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaMemcpyAsync(kmin.data(), s->kappa_min.p, NE * sizeof(double), cudaMemcpyDeviceToHost, st));
    ZCHECK(cudaStreamSynchronize(st));
    bool changed = false;
    for (int e = 0; e < NE; ++e) {
        if (s->P.kappa <= 0.0 && dm[e] < 0.1 * s->P.dhat && dm[e] < W.dmin_last[e]) {
            kap[e] = std::min(2.0 * kap[e], 1e4 * kmin[e]);
            changed = true;
        }
        W.dmin_last[e] = dm[e];
    }
    if (changed) ZCHECK(cudaMemcpyAsync(s->kappa.p, kap.data(), NE * sizeof(double), cudaMemcpyHostToDevice, st));
    s->S.dmin = dm[0];
    s->S.kappa = kap[0];
    s->S.steps += 1;
    ZCHECK(cudaStreamSynchronize(st));
}

// Back to the step's start: x = x^t and the multipliers; with all, also the
// barrier stiffness state (kappa, its flags, d_min) the step may have set
// before it failed.
void restore_step(zema_scene* s, bool all) {
    zema_scene& W = *s;
    cudaStream_t st = s->st;
    size_t n3 = 3 * (size_t)s->n_nodes;
    cudaMemcpyAsync(s->x.p, s->xt.p, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (all && W.kap_save.p) {
        const int NE = s->n_envs;
        cudaMemcpyAsync(s->kappa.p, W.kap_save.p, NE * sizeof(double), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(s->kappa_min.p, W.kap_save.p + NE, NE * sizeof(double), cudaMemcpyDeviceToDevice, st);
        s->kappa_ready = W.kappa_ready_save;
        W.dmin_last = W.dmin_last_save;
        s->first_step_done = W.first_step_done_save;
    }
    if (all && s->n_aff && s->P.al_extrapolate && W.lam_hist.p) {
        // the multipliers before the step's extrapolation
        const size_t na12 = 12 * (size_t)s->n_aff;
        cudaMemcpyAsync(s->lamA.p, W.lam_hist.p, na12 * sizeof(double), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(s->lamA_prev.p, W.lam_hist.p + na12, na12 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    } else if (s->n_aff && W.lam_save.p)
        cudaMemcpyAsync(s->lamA.p, W.lam_save.p, 12 * (size_t)s->n_aff * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (s->G.n_joints && W.lamJ_save.p)
        cudaMemcpyAsync(s->lamJ.p, W.lamJ_save.p, 12 * (size_t)s->G.n_joints * sizeof(double),
                        cudaMemcpyDeviceToDevice, st);
    cudaStreamSynchronize(st);
}

int affine_dev_index(const zema_scene* s, int input_idx) {
    // device affine order = env-major order of input bodies (a stable
    // ordering by env, built once per body count)
    std::vector<int>& m = s->aff_dev_of_input;
    if (m.size() != s->ain.size()) {
        std::vector<int> order(s->ain.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return s->ain[a].env < s->ain[b].env; });
        m.assign(order.size(), -1);
        for (size_t k = 0; k < order.size(); ++k) m[order[k]] = (int)k;
    }
    return input_idx >= 0 && input_idx < (int)m.size() ? m[input_idx] : -1;
}

#define ZEMA_TRY(s)                                  \
    try
#define ZEMA_CATCH(s)                                \
    catch (const ZemaError& e) {                     \
        if (s) (s)->err = e.msg;                     \
        return (zema_status)e.status;                \
    }                                                \
    catch (const std::exception& e) {                \
        if (s) (s)->err = e.what();                  \
        return ZEMA_ERR_OOM;                         \
    }

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

long long zema_launch_count(void) { return zema::launch_counter(); }

void zema_default_params(zema_scene_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->dt = 0.01;
    p->dhat = 1e-3;
    p->kappa = 0.0;
    p->eps_v = 1e-3;
    p->newton_tol_rel = 1e-3;
    p->gravity[1] = -9.81;
    p->pcg_rel_tol = 1e-4;
    p->max_newton = 100;
    p->max_pcg = 10000;
    p->max_al_rounds = 10;
    p->n_envs = 1;
    p->al_extrapolate = 1;
}

zema_status zema_create_scene(const zema_scene_params* params, zema_scene** out) {
    if (!params || !out) return ZEMA_ERR_INVALID_ARG;
    if (!(params->dt > 0) || !(params->dhat > 0) || params->n_envs < 1 || !(params->eps_v > 0) ||
        params->pcg_kind < 0 || params->pcg_kind > 2 || !(params->cell_size < INFINITY))
        return ZEMA_ERR_INVALID_ARG;
    if (params->pcg_cluster_size != 0) {
        // a schedule code: 1..16 (powers of two), + 100, or binned 1001, 1002, 1004, 1101, 1102, 1104
        const int v = params->pcg_cluster_size, low = v % 100;
        const bool uniform = (v < 100 || (v > 100 && v < 200)) && low > 0 && low <= 16 && (low & (low - 1)) == 0;
        const bool binned = v == 1001 || v == 1002 || v == 1004 || v == 1101 || v == 1102 || v == 1104;
        if (!uniform && !binned) return ZEMA_ERR_INVALID_ARG;
    }
    zema_scene* s = new (std::nothrow) zema_scene();
    if (!s) return ZEMA_ERR_OOM;
    s->P = *params;
    s->n_envs = params->n_envs;
    s->st = (cudaStream_t)params->stream;
    s->A.fa = params->alloc;
    s->A.ff = params->free;
    s->A.ctx = params->alloc_ctx;
    s->A.stream = s->st;
    *out = s;
    return ZEMA_OK;
}

zema_status zema_add_tet_body(zema_scene* s, int32_t env, const double* X_rest, int64_t nv, const int32_t* tets,
                              int64_t nt, const double* x0, const double* v0, double E, double nu, double rho,
                              double mu_friction, int32_t* body_id) {
    if (!s) return ZEMA_ERR_INVALID_ARG;
    if (s->finalized) {
        s->err = "bodies must be added before the first step";
        return ZEMA_ERR_STATE;
    }
    if (env < 0 || env >= s->n_envs || !X_rest || !tets || nv < 4 || nt < 1 || !(E > 0) || !(nu > -1 && nu < 0.5) ||
        !(rho > 0) || mu_friction < 0) {
        s->err = "invalid tet body arguments";
        return ZEMA_ERR_INVALID_ARG;
    }
    TetIn B;
    B.env = env;
    B.X.assign(X_rest, X_rest + 3 * nv);
    B.x0 = x0 ? std::vector<double>(x0, x0 + 3 * nv) : B.X;
    B.v0 = v0 ? std::vector<double>(v0, v0 + 3 * nv) : std::vector<double>(3 * nv, 0.0);
    B.T.assign(tets, tets + 4 * nt);
    for (int64_t t = 0; t < nt; ++t) {
        const int* T = &B.T[4 * t];
        for (int k = 0; k < 4; ++k)
            if (T[k] < 0 || T[k] >= nv) {
                s->err = "tet index out of range";
                return ZEMA_ERR_INVALID_ARG;
            }
        const double* a = &B.X[3 * T[0]];
        double e[3][3];
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j) e[k][j] = B.X[3 * T[k + 1] + j] - a[j];
        double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                     e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) + e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
        if (!(det > 0.0)) {
            s->err = "tet with non-positive rest volume";
            return ZEMA_ERR_INVERTED_INPUT;
        }
    }
    B.E = E;
    B.nu = nu;
    B.rho = rho;
    B.mu = mu_friction;
    s->tin.push_back(std::move(B));
    s->bodies.push_back({0, (int)s->tin.size() - 1});
    if (body_id) *body_id = (int32_t)s->bodies.size() - 1;
    return ZEMA_OK;
}

zema_status zema_add_affine_body(zema_scene* s, int32_t env, const double* V_rest, int64_t nv, const int32_t* F,
                                 int64_t nf, const double q0[12], const double qdot0[12], double rho, double stiffness,
                                 double mu_friction, int32_t mode, int32_t* body_id) {
    if (!s) return ZEMA_ERR_INVALID_ARG;
    if (s->finalized) {
        s->err = "bodies must be added before the first step";
        return ZEMA_ERR_STATE;
    }
    if (env < 0 || env >= s->n_envs || !V_rest || !F || !q0 || nv < 4 || nf < 4 || !(rho > 0) || !(stiffness > 0) ||
        mode < 0 || mode > 2 || mu_friction < 0) {
        s->err = "invalid affine body arguments";
        return ZEMA_ERR_INVALID_ARG;
    }
    AffIn B;
    B.env = env;
    B.mode = mode;
    B.V.assign(V_rest, V_rest + 3 * nv);
    B.F.assign(F, F + 3 * nf);
    for (int64_t i = 0; i < 3 * nf; ++i)
        if (B.F[i] < 0 || B.F[i] >= nv) {
            s->err = "face index out of range";
            return ZEMA_ERR_INVALID_ARG;
        }
    // The mass properties integrate over the enclosed volume (Eq. 2), so the
    // surface must be closed and consistently oriented: every directed edge
    // appears once and its reverse once (each edge borders two faces that
    // traverse it in opposite directions), and the signed volume is positive
    // (faces point outward).
    {
        std::vector<uint64_t> de;
        de.reserve(3 * (size_t)nf);
        for (int64_t f = 0; f < nf; ++f)
            for (int k = 0; k < 3; ++k) {
                const uint32_t a = (uint32_t)B.F[3 * f + k], b = (uint32_t)B.F[3 * f + (k + 1) % 3];
                if (a == b) {
                    s->err = "degenerate face in affine body mesh";
                    return ZEMA_ERR_INVALID_ARG;
                }
                de.push_back(((uint64_t)a << 32) | b);
            }
        std::sort(de.begin(), de.end());
        bool ok = std::adjacent_find(de.begin(), de.end()) == de.end();
        for (size_t i = 0; ok && i < de.size(); ++i)
            ok = std::binary_search(de.begin(), de.end(), (de[i] << 32) | (de[i] >> 32));
        if (!ok) {
            s->err = "affine body mesh is not closed and consistently oriented";
            return ZEMA_ERR_INVALID_ARG;
        }
        double vol6 = 0.0;
        for (int64_t f = 0; f < nf; ++f) {
            const double* p0 = &B.V[3 * (size_t)B.F[3 * f]];
            const double* p1 = &B.V[3 * (size_t)B.F[3 * f + 1]];
            const double* p2 = &B.V[3 * (size_t)B.F[3 * f + 2]];
            vol6 += p0[0] * (p1[1] * p2[2] - p1[2] * p2[1]) - p0[1] * (p1[0] * p2[2] - p1[2] * p2[0]) +
                    p0[2] * (p1[0] * p2[1] - p1[1] * p2[0]);
        }
        if (!(vol6 > 0.0)) {
            s->err = "affine body mesh encloses no volume (faces not outward?)";
            return ZEMA_ERR_INVALID_ARG;
        }
    }
    for (int k = 0; k < 12; ++k) {
        B.q0[k] = q0[k];
        B.qd0[k] = qdot0 ? qdot0[k] : 0.0;
    }
    B.rho = rho;
    B.stiff = stiffness;
    B.mu = mu_friction;
    s->ain.push_back(std::move(B));
    s->bodies.push_back({1, (int)s->ain.size() - 1});
    if (body_id) *body_id = (int32_t)s->bodies.size() - 1;
    return ZEMA_OK;
}

zema_status zema_add_prismatic_joint(zema_scene* s, int32_t body1, int32_t body2, const double axis[3],
                                     double kappa, int32_t* joint_id) {
    if (!s) return ZEMA_ERR_INVALID_ARG;
    if (s->finalized) {
        s->err = "joints must be added before the first step";
        return ZEMA_ERR_STATE;
    }
    const int nb = (int)s->bodies.size();
    if (body1 < 0 || body1 >= nb || body2 < 0 || body2 >= nb || body1 == body2 || !axis ||
        s->bodies[body1].first != 1 || s->bodies[body2].first != 1 || !std::isfinite(kappa)) {
        s->err = "a prismatic joint needs two distinct affine bodies and an axis";
        return ZEMA_ERR_INVALID_ARG;
    }
    JointIn J;
    J.a1 = s->bodies[body1].second;
    J.a2 = s->bodies[body2].second;
    const AffIn &B1 = s->ain[J.a1], &B2 = s->ain[J.a2];
    if (B1.env != B2.env || (B1.mode != 0 && B2.mode != 0)) {
        s->err = "jointed bodies must share an env and at least one must be dynamic";
        return ZEMA_ERR_INVALID_ARG;
    }
    const double n = std::sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
    if (!(n > 0.0) || !std::isfinite(n)) {
        s->err = "joint axis must be a nonzero finite vector";
        return ZEMA_ERR_INVALID_ARG;
    }
    for (int i = 0; i < 3; ++i) J.axis[i] = axis[i] / n;
    J.kappa = kappa;
    s->jin.push_back(J);
    if (joint_id) *joint_id = (int32_t)s->jin.size() - 1;
    return ZEMA_OK;
}

zema_status zema_finalize(zema_scene* s) {
    if (s) set_current_stream(s->st);
    if (!s) return ZEMA_ERR_INVALID_ARG;
    if (s->finalized) return ZEMA_OK;
    ZEMA_TRY(s) {
        build(s);
        // reject initial states with touching primitives
        ZL(k_sv_pos, div_up(s->n_sv, TB), TB, 0, s->st)(s->G, s->x.p, s->X.p);
        ZLAUNCH();
        active_pairs(s, s->X.p, true);
        std::vector<double> dm(s->n_envs);
        ZCHECK(cudaMemcpyAsync(dm.data(), s->dmin.p, s->n_envs * sizeof(double), cudaMemcpyDeviceToHost, s->st));
        ZCHECK(cudaStreamSynchronize(s->st));
        for (double d : dm)
            if (!(d > 0.0)) fail(ZEMA_ERR_INTERSECTING_INPUT, "initial state has primitives at distance 0");
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

zema_status zema_set_kinematic_target(zema_scene* s, int32_t body, const double q_target[12]) {
    if (s) set_current_stream(s->st);
    if (!s || !q_target || body < 0 || body >= (int)s->bodies.size() || s->bodies[body].first != 1)
        return ZEMA_ERR_INVALID_ARG;
    ZEMA_TRY(s) {
        int i = s->bodies[body].second;
        if (!s->finalized) {
            // before finalize the target becomes the initial target
            zema_status r = zema_finalize(s);
            if (r != ZEMA_OK) return r;
        }
        int a = affine_dev_index(s, i);
        ZCHECK(cudaMemcpyAsync(s->qtarget.p + 12 * (size_t)a, q_target, 12 * sizeof(double), cudaMemcpyHostToDevice,
                               s->st));
        ZCHECK(cudaStreamSynchronize(s->st));
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

namespace {
// records of 13 doubles: the device affine index, then the 12 target values
__global__ void k_scatter_targets(const double* rec, int n, double* qtarget) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 12 * n) return;
    const int r = i / 12, c = i - 12 * r;
    const int a = (int)rec[13 * (size_t)r];
    qtarget[12 * (size_t)a + c] = rec[13 * (size_t)r + 1 + c];
}
}  // namespace

zema_status zema_set_kinematic_targets(zema_scene* s, int64_t n, const int32_t* bodies, const double* q_targets) {
    if (s) set_current_stream(s->st);
    if (!s || n < 0 || (n > 0 && (!bodies || !q_targets))) return ZEMA_ERR_INVALID_ARG;
    std::vector<char> seen(s->bodies.size(), 0);
    for (int64_t k = 0; k < n; ++k) {
        const int32_t b = bodies[k];
        if (b < 0 || b >= (int)s->bodies.size() || s->bodies[b].first != 1 || seen[b]) return ZEMA_ERR_INVALID_ARG;
        seen[b] = 1;
    }
    if (n == 0) return ZEMA_OK;
    ZEMA_TRY(s) {
        if (!s->finalized) {
            zema_status r = zema_finalize(s);
            if (r != ZEMA_OK) return r;
        }
        const size_t need = 13 * (size_t)n;
        if (!s->kin_ev) ZCHECK(cudaEventCreateWithFlags(&s->kin_ev, cudaEventDisableTiming));
        // the last call's copy out of the staging has run before it is rewritten
        ZCHECK(cudaEventSynchronize(s->kin_ev));
        if (need > s->h_kin_cap) {
            if (s->h_kin) ZCHECK(cudaFreeHost(s->h_kin));
            s->h_kin = nullptr;
            s->h_kin_cap = 0;
            ZCHECK(cudaMallocHost(&s->h_kin, need * sizeof(double)));
            s->h_kin_cap = need;
        }
        for (int64_t k = 0; k < n; ++k) {
            double* r = s->h_kin + 13 * (size_t)k;
            r[0] = (double)affine_dev_index(s, s->bodies[bodies[k]].second);
            std::memcpy(r + 1, q_targets + 12 * (size_t)k, 12 * sizeof(double));
        }
        s->kin_up.ensure(&s->A, need);
        ZCHECK(cudaMemcpyAsync(s->kin_up.p, s->h_kin, need * sizeof(double), cudaMemcpyHostToDevice, s->st));
        ZCHECK(cudaEventRecord(s->kin_ev, s->st));
        ZL(k_scatter_targets, div_up(12 * n, 256), 256, 0, s->st)(s->kin_up.p, (int)n, s->qtarget.p);
        ZLAUNCH();
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

zema_status zema_step(zema_scene* s, int32_t n_steps, zema_step_stats* stats) {
    if (s) set_current_stream(s->st);
    if (!s || n_steps < 0) return ZEMA_ERR_INVALID_ARG;
    if (!s->finalized) {
        zema_status r = zema_finalize(s);
        if (r != ZEMA_OK) return r;
    }
    std::memset(&s->S, 0, sizeof(s->S));
    s->S.dmin = INFINITY;
    s->newton_count = 0;
    zema_status status = ZEMA_OK;
    for (int k = 0; k < n_steps; ++k) {
        try {
            do_step(s);
        } catch (const ZemaError& e) {
            s->err = e.msg;
            status = (zema_status)e.status;
            s->fault_armed = 0;
            restore_step(s);
            break;
        }
    }
    s->fault_armed = 0;
    if (stats) *stats = s->S;
    return status;
}

zema_status zema_get_state(const zema_scene* cs, int32_t body, double* out, int64_t cap, int64_t* written) {
    zema_scene* s = const_cast<zema_scene*>(cs);
    if (!s || !out || body < 0 || body >= (int)s->bodies.size()) return ZEMA_ERR_INVALID_ARG;
    ZEMA_TRY(s) {
        auto bk = s->bodies[body];
        if (bk.first == 0) {
            const TetIn& B = s->tin[bk.second];
            int64_t nv = (int64_t)B.X.size() / 3;
            if (cap < 6 * nv) return ZEMA_ERR_INVALID_ARG;
            if (!s->finalized) {
                std::copy(B.x0.begin(), B.x0.end(), out);
                std::copy(B.v0.begin(), B.v0.end(), out + 3 * nv);
            } else {
                size_t n0 = s->tet_body_node0[bk.second];
                ZCHECK(cudaMemcpyAsync(out, s->x.p + 3 * n0, 3 * nv * sizeof(double), cudaMemcpyDeviceToHost, s->st));
                ZCHECK(cudaMemcpyAsync(out + 3 * nv, s->v.p + 3 * n0, 3 * nv * sizeof(double), cudaMemcpyDeviceToHost,
                                       s->st));
                ZCHECK(cudaStreamSynchronize(s->st));
            }
            if (written) *written = 6 * nv;
            return ZEMA_OK;
        }
        if (cap < 24) return ZEMA_ERR_INVALID_ARG;
        const AffIn& B = s->ain[bk.second];
        if (!s->finalized) {
            for (int k = 0; k < 12; ++k) {
                out[k] = B.q0[k];
                out[12 + k] = B.qd0[k];
            }
        } else {
            double xc[12], vc[12];
            size_t n0 = s->aff_node0_h[bk.second];
            ZCHECK(cudaMemcpyAsync(xc, s->x.p + 3 * n0, 12 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
            ZCHECK(cudaMemcpyAsync(vc, s->v.p + 3 * n0, 12 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
            ZCHECK(cudaStreamSynchronize(s->st));
            const double* c = &s->aff_com_h[3 * bk.second];
            for (int i = 0; i < 3; ++i) {
                // A_ik = c_k[i]; p = p' - A com
                double Ac = 0.0, Adc = 0.0;
                for (int k = 0; k < 3; ++k) {
                    out[3 + 3 * i + k] = xc[3 * (1 + k) + i];
                    out[12 + 3 + 3 * i + k] = vc[3 * (1 + k) + i];
                    Ac += xc[3 * (1 + k) + i] * c[k];
                    Adc += vc[3 * (1 + k) + i] * c[k];
                }
                out[i] = xc[i] - Ac;
                out[12 + i] = vc[i] - Adc;
            }
        }
        if (written) *written = 24;
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

zema_status zema_set_state(zema_scene* s, int32_t body, const double* in, int64_t n) {
    if (!s || !in || body < 0 || body >= (int)s->bodies.size()) return ZEMA_ERR_INVALID_ARG;
    ZEMA_TRY(s) {
        auto bk = s->bodies[body];
        if (bk.first == 0) {
            TetIn& B = s->tin[bk.second];
            int64_t nv = (int64_t)B.X.size() / 3;
            if (n != 6 * nv) return ZEMA_ERR_INVALID_ARG;
            if (!s->finalized) {
                std::copy(in, in + 3 * nv, B.x0.begin());
                std::copy(in + 3 * nv, in + 6 * nv, B.v0.begin());
                return ZEMA_OK;
            }
            size_t n0 = s->tet_body_node0[bk.second];
            ZCHECK(cudaMemcpyAsync(s->x.p + 3 * n0, in, 3 * nv * sizeof(double), cudaMemcpyHostToDevice, s->st));
            ZCHECK(cudaMemcpyAsync(s->v.p + 3 * n0, in + 3 * nv, 3 * nv * sizeof(double), cudaMemcpyHostToDevice, s->st));
            ZCHECK(cudaStreamSynchronize(s->st));
            return ZEMA_OK;
        }
        if (n != 24) return ZEMA_ERR_INVALID_ARG;
        AffIn& B = s->ain[bk.second];
        if (!s->finalized) {
            for (int k = 0; k < 12; ++k) {
                B.q0[k] = in[k];
                B.qd0[k] = in[12 + k];
            }
            return ZEMA_OK;
        }
        double xc[12], vc[12];
        const double* c = &s->aff_com_h[3 * bk.second];
        bool fixed = B.mode == 1;
        for (int i = 0; i < 3; ++i) {
            double Ac = 0.0, Adc = 0.0;
            for (int k = 0; k < 3; ++k) {
                xc[3 * (1 + k) + i] = in[3 + 3 * i + k];
                vc[3 * (1 + k) + i] = fixed ? 0.0 : in[12 + 3 + 3 * i + k];
                Ac += in[3 + 3 * i + k] * c[k];
                Adc += in[12 + 3 + 3 * i + k] * c[k];
            }
            xc[i] = in[i] + Ac;
            vc[i] = fixed ? 0.0 : in[12 + i] + Adc;
        }
        size_t n0 = s->aff_node0_h[bk.second];
        ZCHECK(cudaMemcpyAsync(s->x.p + 3 * n0, xc, 12 * sizeof(double), cudaMemcpyHostToDevice, s->st));
        ZCHECK(cudaMemcpyAsync(s->v.p + 3 * n0, vc, 12 * sizeof(double), cudaMemcpyHostToDevice, s->st));
        ZCHECK(cudaStreamSynchronize(s->st));
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

}  // extern "C"

namespace {
// The flat state of every body in order of addition (the layout of
// zema_get_state, bodies back to back) to (set) or from (get) the node
// arrays.  One block per body: a tet body's vertices (x then v) by the
// block's threads; an affine body's 24 values by thread 0 (caller's frame
// q = (p, A by rows) against the internal p' = p + A com and columns of A).
template <bool kSet>
__global__ void k_scene_state(int n_bodies, const int* node0, const int* nv, const int64_t* off, const int* fixed,
                              const double* com, double* x, double* v, double* flat) {
    const int b = blockIdx.x;
    if (b >= n_bodies) return;
    const int n0 = node0[b], m = nv[b];
    double* f = flat + off[b];
    if (m >= 0) {
        for (int i = threadIdx.x; i < 3 * m; i += blockDim.x) {
            if (kSet) {
                x[3 * (size_t)n0 + i] = f[i];
                v[3 * (size_t)n0 + i] = f[3 * (size_t)m + i];
            } else {
                f[i] = x[3 * (size_t)n0 + i];
                f[3 * (size_t)m + i] = v[3 * (size_t)n0 + i];
            }
        }
        return;
    }
    if (threadIdx.x != 0) return;
    const double* c = com + 3 * (size_t)b;
    double* xc = x + 3 * (size_t)n0;
    double* vc = v + 3 * (size_t)n0;
    for (int i = 0; i < 3; ++i) {
        double Ac = 0.0, Adc = 0.0;
        for (int k = 0; k < 3; ++k) {
            if (kSet) {
                xc[3 * (1 + k) + i] = f[3 + 3 * i + k];
                vc[3 * (1 + k) + i] = fixed[b] ? 0.0 : f[12 + 3 + 3 * i + k];
                Ac += f[3 + 3 * i + k] * c[k];
                Adc += f[12 + 3 + 3 * i + k] * c[k];
            } else {
                f[3 + 3 * i + k] = xc[3 * (1 + k) + i];
                f[12 + 3 + 3 * i + k] = vc[3 * (1 + k) + i];
                Ac += xc[3 * (1 + k) + i] * c[k];
                Adc += vc[3 * (1 + k) + i] * c[k];
            }
        }
        if (kSet) {
            xc[i] = f[i] + Ac;
            vc[i] = fixed[b] ? 0.0 : f[12 + i] + Adc;
        } else {
            f[i] = xc[i] - Ac;
            f[12 + i] = vc[i] - Adc;
        }
    }
}

// the per-body tables of the flat scene state (built once)
int64_t scene_state_tables(zema_scene* s) {
    if (s->sst_n >= 0) return s->sst_n;
    const int nb = (int)s->bodies.size();
    std::vector<int> node0(nb), nv(nb), fixed(nb, 0);
    std::vector<int64_t> off(nb);
    std::vector<double> com(3 * (size_t)nb, 0.0);
    int64_t o = 0;
    for (int b = 0; b < nb; ++b) {
        const auto bk = s->bodies[b];
        off[b] = o;
        if (bk.first == 0) {
            node0[b] = s->tet_body_node0[bk.second];
            nv[b] = (int)(s->tin[bk.second].X.size() / 3);
            o += 6 * (int64_t)nv[b];
        } else {
            node0[b] = s->aff_node0_h[bk.second];
            nv[b] = -1;
            fixed[b] = s->ain[bk.second].mode == 1 ? 1 : 0;
            for (int k = 0; k < 3; ++k) com[3 * (size_t)b + k] = s->aff_com_h[3 * (size_t)bk.second + k];
            o += 24;
        }
    }
    up(s, s->sst_node0, node0);
    up(s, s->sst_nv, nv);
    up(s, s->sst_fixed, fixed);
    up(s, s->sst_off, off);
    up(s, s->sst_com, com);
    s->sst_buf.ensure(&s->A, (size_t)o + 1);
    s->sst_n = o;
    return o;
}
}  // namespace

extern "C" {

zema_status zema_scene_state_size(const zema_scene* cs, int64_t* n) {
    zema_scene* s = const_cast<zema_scene*>(cs);
    if (!s || !n) return ZEMA_ERR_INVALID_ARG;
    if (!s->finalized) return ZEMA_ERR_STATE;
    ZEMA_TRY(s) {
        *n = scene_state_tables(s);
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

zema_status zema_get_scene_state(const zema_scene* cs, double* out, int64_t cap, int64_t* written) {
    zema_scene* s = const_cast<zema_scene*>(cs);
    if (s) set_current_stream(s->st);
    if (!s || !out) return ZEMA_ERR_INVALID_ARG;
    if (!s->finalized) return ZEMA_ERR_STATE;
    ZEMA_TRY(s) {
        const int64_t n = scene_state_tables(s);
        if (cap < n) return ZEMA_ERR_INVALID_ARG;
        const int nb = (int)s->bodies.size();
        if (nb)
            ZL(k_scene_state<false>, nb, 128, 0, s->st)(nb, s->sst_node0.p, s->sst_nv.p, s->sst_off.p,
                                                        s->sst_fixed.p, s->sst_com.p, s->x.p, s->v.p, s->sst_buf.p);
        ZLAUNCH();
        ZCHECK(cudaMemcpyAsync(out, s->sst_buf.p, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s->st));
        ZCHECK(cudaStreamSynchronize(s->st));
        if (written) *written = n;
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

zema_status zema_set_scene_state(zema_scene* s, const double* in, int64_t n) {
    if (s) set_current_stream(s->st);
    if (!s || !in) return ZEMA_ERR_INVALID_ARG;
    if (!s->finalized) return ZEMA_ERR_STATE;
    ZEMA_TRY(s) {
        if (n != scene_state_tables(s)) return ZEMA_ERR_INVALID_ARG;
        const int nb = (int)s->bodies.size();
        ZCHECK(cudaMemcpyAsync(s->sst_buf.p, in, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s->st));
        if (nb)
            ZL(k_scene_state<true>, nb, 128, 0, s->st)(nb, s->sst_node0.p, s->sst_nv.p, s->sst_off.p, s->sst_fixed.p,
                                                       s->sst_com.p, s->x.p, s->v.p, s->sst_buf.p);
        ZLAUNCH();
        // the caller may reuse `in` on return
        ZCHECK(cudaStreamSynchronize(s->st));
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

zema_status zema_copy_soft_state_device(const zema_scene* cs, double* x_dev, double* v_dev) {
    zema_scene* s = const_cast<zema_scene*>(cs);
    if (!s || !s->finalized) return ZEMA_ERR_STATE;
    ZEMA_TRY(s) {
        size_t off = 0;
        for (size_t i = 0; i < s->tin.size(); ++i) {
            size_t nv = s->tin[i].X.size() / 3;
            size_t n0 = s->tet_body_node0[i];
            if (x_dev)
                ZCHECK(cudaMemcpyAsync(x_dev + 3 * off, s->x.p + 3 * n0, 3 * nv * sizeof(double), cudaMemcpyDeviceToDevice,
                                       s->st));
            if (v_dev)
                ZCHECK(cudaMemcpyAsync(v_dev + 3 * off, s->v.p + 3 * n0, 3 * nv * sizeof(double), cudaMemcpyDeviceToDevice,
                                       s->st));
            off += nv;
        }
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

zema_status zema_scene_counts(const zema_scene* s, int64_t out[8]) {
    if (!s || !out) return ZEMA_ERR_INVALID_ARG;
    int64_t nv = 0, nt = 0;
    for (auto& b : s->tin) {
        nv += (int64_t)b.X.size() / 3;
        nt += (int64_t)b.T.size() / 4;
    }
    out[0] = nv;
    out[1] = nt;
    out[2] = (int64_t)s->ain.size();
    out[3] = s->n_sv;
    out[4] = s->n_edges;
    out[5] = s->n_tris;
    out[6] = s->n_nodes;
    out[7] = s->n_envs;
    return ZEMA_OK;
}

zema_status zema_get_kappa(const zema_scene* cs, int32_t env, double* kappa) {
    zema_scene* s = const_cast<zema_scene*>(cs);
    if (!s || !kappa || env < 0 || env >= s->n_envs || !s->finalized) return ZEMA_ERR_INVALID_ARG;
    ZEMA_TRY(s) {
        ZCHECK(cudaMemcpyAsync(kappa, s->kappa.p + env, sizeof(double), cudaMemcpyDeviceToHost, s->st));
        ZCHECK(cudaStreamSynchronize(s->st));
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

zema_status zema_set_kappa(zema_scene* s, int32_t env, double kappa, double kappa_min) {
    if (!s || env < 0 || env >= s->n_envs || !(kappa > 0) || !(kappa_min > 0)) return ZEMA_ERR_INVALID_ARG;
    if (!s->finalized) {
        zema_status r = zema_finalize(s);
        if (r != ZEMA_OK) return r;
    }
    ZEMA_TRY(s) {
        ZCHECK(cudaMemcpyAsync(s->kappa.p + env, &kappa, sizeof(double), cudaMemcpyHostToDevice, s->st));
        ZCHECK(cudaMemcpyAsync(s->kappa_min.p + env, &kappa_min, sizeof(double), cudaMemcpyHostToDevice, s->st));
        ZCHECK(cudaStreamSynchronize(s->st));
        s->kappa_ready[env] = 1;
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

// Whole-scene checkpoint: every quantity that carries over from one time
// step to the next (Eq. 11 state, kinematic targets and augmented-Lagrangian
// multipliers of Eq. 13, the per-env barrier stiffness and the d_min of the
// stiffness rule).  Layout: 8 uint64 header words (magic, version, nodes,
// affine bodies, joints, envs, first step done, 0), then doubles: x and v (3
// per node), q~ and lambda_A (12 per affine body), lambda of the joints (12
// each), kappa, kappa_min, last d_min and kappa-set flag (one per env).
constexpr uint64_t kCkptMagic = 0x31504B43414D455Aull;  // "ZEMACKP1"
constexpr uint64_t kCkptVersion = 2;  // 2: with the kinematic multipliers of the step before

size_t ckpt_doubles(const zema_scene* s) {
    return 6 * (size_t)s->n_nodes + 36 * (size_t)s->n_aff + 12 * (size_t)s->G.n_joints + 4 * (size_t)s->n_envs;
}

zema_status zema_checkpoint_size(const zema_scene* s, int64_t* bytes) {
    if (!s || !bytes) return ZEMA_ERR_INVALID_ARG;
    if (!s->finalized) return ZEMA_ERR_STATE;
    *bytes = (int64_t)(8 * sizeof(uint64_t) + ckpt_doubles(s) * sizeof(double));
    return ZEMA_OK;
}

zema_status zema_save_checkpoint(const zema_scene* cs, void* buf, int64_t cap, int64_t* written) {
    zema_scene* s = const_cast<zema_scene*>(cs);
    if (!s || !buf) return ZEMA_ERR_INVALID_ARG;
    if (!s->finalized) return ZEMA_ERR_STATE;
    const size_t nd = ckpt_doubles(s), bytes = 8 * sizeof(uint64_t) + nd * sizeof(double);
    if (cap < (int64_t)bytes) return ZEMA_ERR_INVALID_ARG;
    ZEMA_TRY(s) {
        uint64_t* h = (uint64_t*)buf;
        const int NE = s->n_envs, NA = s->n_aff, NJ = s->G.n_joints;
        const size_t n3 = 3 * (size_t)s->n_nodes;
        h[0] = kCkptMagic;
        h[1] = kCkptVersion;
        h[2] = (uint64_t)s->n_nodes;
        h[3] = (uint64_t)NA;
        h[4] = (uint64_t)NJ;
        h[5] = (uint64_t)NE;
        h[6] = s->first_step_done ? 1 : 0;
        h[7] = 0;
        double* d = (double*)(h + 8);
        cudaStream_t st = s->st;
        ZCHECK(cudaMemcpyAsync(d, s->x.p, n3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        ZCHECK(cudaMemcpyAsync(d + n3, s->v.p, n3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        d += 2 * n3;
        if (NA) {
            ZCHECK(cudaMemcpyAsync(d, s->qtarget.p, 12 * (size_t)NA * sizeof(double), cudaMemcpyDeviceToHost, st));
            ZCHECK(cudaMemcpyAsync(d + 12 * (size_t)NA, s->lamA.p, 12 * (size_t)NA * sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
            ZCHECK(cudaMemcpyAsync(d + 24 * (size_t)NA, s->lamA_prev.p, 12 * (size_t)NA * sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
        }
        d += 36 * (size_t)NA;
        if (NJ) ZCHECK(cudaMemcpyAsync(d, s->lamJ.p, 12 * (size_t)NJ * sizeof(double), cudaMemcpyDeviceToHost, st));
        d += 12 * (size_t)NJ;
        ZCHECK(cudaMemcpyAsync(d, s->kappa.p, NE * sizeof(double), cudaMemcpyDeviceToHost, st));
        ZCHECK(cudaMemcpyAsync(d + NE, s->kappa_min.p, NE * sizeof(double), cudaMemcpyDeviceToHost, st));
        ZCHECK(cudaStreamSynchronize(st));
        for (int e = 0; e < NE; ++e) {
            d[2 * NE + e] = e < (int)s->dmin_last.size() ? s->dmin_last[e] : INFINITY;
            d[3 * NE + e] = s->kappa_ready[e] ? 1.0 : 0.0;
        }
        if (written) *written = (int64_t)bytes;
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

zema_status zema_load_checkpoint(zema_scene* s, const void* buf, int64_t bytes) {
    if (!s || !buf || bytes < (int64_t)(8 * sizeof(uint64_t))) return ZEMA_ERR_INVALID_ARG;
    if (!s->finalized) {
        zema_status r = zema_finalize(s);
        if (r != ZEMA_OK) return r;
    }
    const uint64_t* h = (const uint64_t*)buf;
    const int NE = s->n_envs, NA = s->n_aff, NJ = s->G.n_joints;
    if (h[0] != kCkptMagic || h[1] != kCkptVersion || h[2] != (uint64_t)s->n_nodes || h[3] != (uint64_t)NA ||
        h[4] != (uint64_t)NJ || h[5] != (uint64_t)NE)
        return ZEMA_ERR_INVALID_ARG;
    if (bytes != (int64_t)(8 * sizeof(uint64_t) + ckpt_doubles(s) * sizeof(double))) return ZEMA_ERR_INVALID_ARG;
    const double* d = (const double*)(h + 8);
    const size_t n3 = 3 * (size_t)s->n_nodes;
    for (size_t i = 0; i < 2 * n3; ++i)
        if (!std::isfinite(d[i])) return ZEMA_ERR_INVALID_ARG;
    for (int e = 0; e < NE; ++e) {
        const double* k = d + 2 * n3 + 36 * (size_t)NA + 12 * (size_t)NJ;
        if (!(k[e] >= 0.0 && k[e] < INFINITY) || !(k[NE + e] >= 0.0 && k[NE + e] < INFINITY))
            return ZEMA_ERR_INVALID_ARG;
    }
    ZEMA_TRY(s) {
        cudaStream_t st = s->st;
        ZCHECK(cudaMemcpyAsync(s->x.p, d, n3 * sizeof(double), cudaMemcpyHostToDevice, st));
        ZCHECK(cudaMemcpyAsync(s->v.p, d + n3, n3 * sizeof(double), cudaMemcpyHostToDevice, st));
        d += 2 * n3;
        if (NA) {
            ZCHECK(cudaMemcpyAsync(s->qtarget.p, d, 12 * (size_t)NA * sizeof(double), cudaMemcpyHostToDevice, st));
            ZCHECK(cudaMemcpyAsync(s->lamA.p, d + 12 * (size_t)NA, 12 * (size_t)NA * sizeof(double),
                                   cudaMemcpyHostToDevice, st));
            ZCHECK(cudaMemcpyAsync(s->lamA_prev.p, d + 24 * (size_t)NA, 12 * (size_t)NA * sizeof(double),
                                   cudaMemcpyHostToDevice, st));
        }
        d += 36 * (size_t)NA;
        if (NJ) ZCHECK(cudaMemcpyAsync(s->lamJ.p, d, 12 * (size_t)NJ * sizeof(double), cudaMemcpyHostToDevice, st));
        d += 12 * (size_t)NJ;
        ZCHECK(cudaMemcpyAsync(s->kappa.p, d, NE * sizeof(double), cudaMemcpyHostToDevice, st));
        ZCHECK(cudaMemcpyAsync(s->kappa_min.p, d + NE, NE * sizeof(double), cudaMemcpyHostToDevice, st));
        ZCHECK(cudaStreamSynchronize(st));
        s->first_step_done = h[6] != 0;
        s->dmin_last.assign(d + 2 * NE, d + 3 * NE);
        for (int e = 0; e < NE; ++e) s->kappa_ready[e] = d[3 * NE + e] != 0.0 ? 1 : 0;
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

zema_status zema_inject_fault(zema_scene* s, int32_t kind, int32_t newton_iter) {
    if (!s || kind < ZEMA_FAULT_NONE || kind > ZEMA_FAULT_NO_DECREASE || newton_iter < 0) return ZEMA_ERR_INVALID_ARG;
    ZEMA_TRY(s) {
        s->fault_dev.ensure(&s->A, 2);
        ZCHECK(cudaMemsetAsync(s->fault_dev.p, 0, 2 * sizeof(int), s->st));
        ZCHECK(cudaStreamSynchronize(s->st));
        s->fault_kind = kind;
        s->fault_at = newton_iter;
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

zema_status zema_load_warmstart(zema_scene* s, const void* blob, int64_t bytes) {
    if (!s || !blob || bytes < 12) return ZEMA_ERR_INVALID_ARG;
    const uint32_t* h = (const uint32_t*)blob;
    if (h[0] != 0x5357455Au) return ZEMA_ERR_INVALID_ARG;
    const uint32_t L = h[1];
    if (L < 1 || L > 16 || bytes < (int64_t)(4 * (L + 3))) return ZEMA_ERR_INVALID_ARG;
    std::vector<int> dims(L + 1);
    for (uint32_t l = 0; l <= L; ++l) dims[l] = (int)h[2 + l];
    const bool per_body = dims[0] == kWsAffFeatures && dims[L] == kWsAffOutputs;
    if (!per_body && (dims[0] != kWsFeatures || dims[L] != kWsOutputs)) return ZEMA_ERR_INVALID_ARG;
    size_t np = 0;
    for (uint32_t l = 0; l < L; ++l) {
        if (dims[l] < 1 || dims[l] > 4096 || dims[l + 1] < 1 || dims[l + 1] > 4096) return ZEMA_ERR_INVALID_ARG;
        np += (size_t)dims[l] * dims[l + 1] + dims[l + 1];
    }
    if (bytes != (int64_t)(4 * (L + 3) + 4 * np)) return ZEMA_ERR_INVALID_ARG;
    ZEMA_TRY(s) {
        Mlp* net = new Mlp(dims, 0, s->st);
        const float* th = (const float*)(h + 3 + L);
        ZCHECK(cudaMemcpyAsync(net->theta.p, th, np * sizeof(float), cudaMemcpyHostToDevice, s->st));
        net->refresh_bf16();
        ZCHECK(cudaStreamSynchronize(s->st));
        Mlp*& slot = per_body ? s->ws_anet : s->ws_net;
        delete slot;
        slot = net;
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

zema_status zema_record_warmstart(zema_scene* s, float* features, float* targets, int64_t cap_rows) {
    if (!s || (features == nullptr) != (targets == nullptr)) return ZEMA_ERR_INVALID_ARG;
    if (!s->finalized) {
        zema_status r = zema_finalize(s);
        if (r != ZEMA_OK) return r;
    }
    if (features && cap_rows < s->ws_ns) return ZEMA_ERR_INVALID_ARG;
    s->rec_feat = features;
    s->rec_targ = targets;
    return ZEMA_OK;
}

zema_status zema_set_material(zema_scene* s, int32_t body, int32_t model) {
    if (!s || body < 0 || body >= (int)s->bodies.size() || s->bodies[body].first != 0 || model < 0 || model > 2)
        return ZEMA_ERR_INVALID_ARG;
    if (s->finalized) return ZEMA_ERR_INVALID_ARG;
    s->tin[s->bodies[body].second].model = model;
    return ZEMA_OK;
}

zema_status zema_set_springs(zema_scene* s, int32_t body, const int32_t* verts, int64_t n, const double* targets,
                             double k) {
    if (s) set_current_stream(s->st);
    if (!s || body < 0 || body >= (int)s->bodies.size() || s->bodies[body].first != 0 || n < 0 ||
        (n > 0 && (!verts || !targets)) || !(k >= 0.0) || !std::isfinite(k))
        return ZEMA_ERR_INVALID_ARG;
    const int tb = s->bodies[body].second;
    TetIn& B = s->tin[tb];
    const int nv = (int)(B.X.size() / 3);
    for (int64_t i = 0; i < n; ++i) {
        if (verts[i] < 0 || verts[i] >= nv) return ZEMA_ERR_INVALID_ARG;
        for (int j = 0; j < 3; ++j)
            if (!std::isfinite(targets[3 * i + j])) return ZEMA_ERR_INVALID_ARG;
    }
    B.spring_v.assign(verts, verts + n);
    B.spring_x.assign(targets, targets + 3 * n);
    B.spring_k = n > 0 ? k : 0.0;
    if (!s->finalized) return ZEMA_OK;
    ZEMA_TRY(s) {
        upload_springs(s, tb);
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

zema_status zema_contact_forces(zema_scene* s, double* forces, int64_t cap) {
    if (s) set_current_stream(s->st);
    if (!s || !forces || cap < 3 * (int64_t)s->bodies.size()) return ZEMA_ERR_INVALID_ARG;
    if (!s->finalized) {
        zema_status r = zema_finalize(s);
        if (r != ZEMA_OK) return r;
    }
    ZEMA_TRY(s) {
        cudaStream_t st = s->st;
        const int nb = (int)s->bodies.size();
        if (s->body_env.cap == 0) {
            std::vector<int> be(nb);
            for (int b = 0; b < nb; ++b)
                be[b] = s->bodies[b].first == 0 ? s->tin[s->bodies[b].second].env : s->ain[s->bodies[b].second].env;
            up(s, s->body_env, be);
        }
        s->body_force.ensure(&s->A, 3 * (size_t)nb + 3);
        // active pairs at the current positions (fresh broad phase)
        ZL(k_sv_pos, div_up(s->n_sv, TB), TB, 0, st)(s->G, s->x.p, s->X.p);
        ZLAUNCH();
        active_pairs(s, s->X.p, false);
        ZL(k_body_contact_force, nb, 128, 0, st)(s->G, s->X.p, s->act.p, s->act_env.p, s->body_env.p, s->kappa.p,
                                                1.0 / (s->P.dt * s->P.dt), s->body_force.p);
        ZLAUNCH();
        ZCHECK(cudaMemcpyAsync(forces, s->body_force.p, 3 * (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, st));
        ZCHECK(cudaStreamSynchronize(st));
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

zema_status zema_record_warmstart_affine(zema_scene* s, float* features, float* targets, int64_t cap_rows) {
    if (!s || (features == nullptr) != (targets == nullptr)) return ZEMA_ERR_INVALID_ARG;
    if (!s->finalized) {
        zema_status r = zema_finalize(s);
        if (r != ZEMA_OK) return r;
    }
    if (features && cap_rows < s->ws_na) return ZEMA_ERR_INVALID_ARG;
    s->rec_afeat = features;
    s->rec_atarg = targets;
    return ZEMA_OK;
}

zema_status zema_autotune(zema_scene* s) {
    if (!s) return ZEMA_ERR_INVALID_ARG;
    // a pinned cluster size is kept
    s->pcgc_tune[0] = s->pcgc_tune[1] = s->P.pcg_cluster_size <= 0;
    return ZEMA_OK;
}

zema_status zema_get_tuning(const zema_scene* s, int32_t precision, int32_t* cluster_size, int32_t* cand,
                            float* ms, int32_t cap, int32_t* n) {
    if (!s || !cluster_size || precision < 0 || precision > 1) return ZEMA_ERR_INVALID_ARG;
    *cluster_size = s->pcgc_cs[precision];
    const auto& t = s->pcgc_tuned[precision];
    if (n) *n = (int32_t)t.size();
    for (int i = 0; i < (int)t.size() && i < cap; ++i) {
        if (cand) cand[i] = t[i].first;
        if (ms) ms[i] = t[i].second;
    }
    return ZEMA_OK;
}

const char* zema_last_error(const zema_scene* s) { return s ? s->err.c_str() : "null scene"; }

void zema_destroy_scene(zema_scene* s) {
    if (!s) return;
    if (s->st) cudaStreamSynchronize(s->st);
    delete s;
}

zema_status zema_eval_energy_grad(zema_scene* s, int32_t apply_predictor, double* energy_out, double* grad) {
    if (s) set_current_stream(s->st);
    if (!s || !energy_out) return ZEMA_ERR_INVALID_ARG;
    if (!s->finalized) {
        zema_status r = zema_finalize(s);
        if (r != ZEMA_OK) return r;
    }
    ZEMA_TRY(s) {
        cudaStream_t st = s->st;
        Geo& G = s->G;
        int NE = s->n_envs;
        if (apply_predictor) {
            const double* gr = s->P.gravity;
            ZL(k_predict, div_up(s->n_nodes, TB), TB, 0, st)(G, s->x.p, s->v.p, s->xt.p, s->xhat.p, gr[0], gr[1], gr[2]);
            if (s->n_aff) ZL(k_predict_affine, div_up(s->n_aff, 64), 64, 0, st)(G, s->xhat.p, gr[0], gr[1], gr[2]);
            ZLAUNCH();
            init_kappa(s);
            lag_friction(s);
        }
        ZL(k_sv_pos, div_up(s->n_sv, TB), TB, 0, st)(G, s->x.p, s->X.p);
        ZLAUNCH();
        active_pairs(s, s->X.p, false);
        energy(s, s->x.p, s->cand.p, s->m_env.p);
        for (int e = 0; e < NE; ++e) energy_out[e] = s->hd[e];
        if (grad) {
            grad_hess(s, true, true, false);
            ZL(k_affine_grad_to_row, div_up(s->n_aff + 1, 64), 64, 0, st)(G, s->g.p);
            ZLAUNCH();
            std::vector<double> gh(3 * (size_t)s->n_nodes);
            ZCHECK(cudaMemcpyAsync(gh.data(), s->g.p, gh.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
            ZCHECK(cudaStreamSynchronize(st));
            size_t o = 0;
            for (size_t b = 0; b < s->bodies.size(); ++b) {
                auto bk = s->bodies[b];
                if (bk.first == 0) {
                    size_t nv = s->tin[bk.second].X.size() / 3, n0 = s->tet_body_node0[bk.second];
                    for (size_t k = 0; k < 3 * nv; ++k) grad[o + k] = gh[3 * n0 + k];
                    o += 3 * nv;
                } else {
                    size_t n0 = s->aff_node0_h[bk.second];
                    for (int k = 0; k < 12; ++k) grad[o + k] = s->ain[bk.second].mode == 1 ? 0.0 : gh[3 * n0 + k];
                    o += 12;
                }
            }
        }
        return ZEMA_OK;
    }
    ZEMA_CATCH(s)
}

}  // extern "C"

// ===========================================================================
// Stand-alone entry points on host arrays (same device code as the stepper)
// ===========================================================================
namespace {

struct Temp {
    Allocator A;
    std::vector<std::pair<void*, size_t>> bufs;
    cudaStream_t st;
    explicit Temp(cudaStream_t s) : st(s) { A.stream = s; }
    template <class T>
    T* put(const T* h, size_t n) {
        T* d = (T*)A.get(n * sizeof(T) + 16);
        bufs.push_back({d, n * sizeof(T) + 16});
        if (h && n) ZCHECK(cudaMemcpyAsync(d, h, n * sizeof(T), cudaMemcpyHostToDevice, st));
        return d;
    }
    ~Temp() {
        for (auto& b : bufs) A.put(b.first, b.second);
    }
};

__global__ void k_sv_env_of(const int* sv_body, const int* b_env, int n, int* sv_env) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) sv_env[i] = b_env[sv_body[i]];
}

// the scene's barrier kernels (the two-launch form) on caller stencils (kappa = 1)
__global__ void __launch_bounds__(kRawThreads) k_local_barrier(const double* x12, const int* is_ee,
                                                              const double* eps_x, int n, double dhat, double* e_out,
                                                              double* g_out, double* H_out, int* flag) {
    auto load = [&](int i, V3* x, int& ee, double& eps, double& kap) {
        for (int k = 0; k < 4; ++k) x[k] = ld3(x12 + 12 * (size_t)i + 3 * k);
        ee = is_ee[i];
        eps = eps_x[i];
        kap = 1.0;
    };
    barrier_gh_raw<double>(n, load, dhat, H_out, g_out, e_out, flag);
}

__global__ void __launch_bounds__(kCoopLanes * kProjPairs) k_local_project(int n, const int* flag, double* H_out) {
    barrier_project_half<double>(n, 1.0, flag, H_out);
}

__global__ void k_local_distance(const double* x12, const int* is_ee, int n, double* d2, double* w) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    V3 x[4];
    for (int k = 0; k < 4; ++k) x[k] = ld3(x12 + 12 * (size_t)i + 3 * k);
    DistInfo di = classify(x, is_ee[i] != 0);
    d2[i] = di.d2;
    for (int k = 0; k < 4; ++k) w[4 * (size_t)i + k] = di.w[k];
}

__global__ void __launch_bounds__(EL_T) k_local_nh(const double* F9, int n, double mu, double lam, double* psi,
                                                   double* g, double* H) {
    extern __shared__ double sm[];
    int i = blockIdx.x * EL_T + threadIdx.x;
    if (i >= n) return;
    SMat<9> M{sm + threadIdx.x, EL_T};
    double P[9], ps;
    if (!nh_eval(F9 + 9 * (size_t)i, mu, lam, ps, P, nullptr)) {
        psi[i] = INFINITY;
        return;
    }
    nh_hessian_projected<double>(F9 + 9 * (size_t)i, mu, lam, M);
    psi[i] = ps;
    for (int a = 0; a < 9; ++a) {
        g[9 * (size_t)i + a] = P[a];
        for (int b = 0; b < 9; ++b) H[81 * (size_t)i + 9 * a + b] = M(a, b);
    }
}

// any material: density, first Piola stress and PSD-projected F-space Hessian
__global__ void __launch_bounds__(EL_T) k_local_elastic(const double* F9, int n, double mu, double lam, int model,
                                                        double* psi, double* g, double* H) {
    extern __shared__ double sm[];
    int i = blockIdx.x * EL_T + threadIdx.x;
    if (i >= n) return;
    SMat<9> M{sm + threadIdx.x, EL_T};
    const double* F = F9 + 9 * (size_t)i;
    double P[9], ps, W[81];
    bool ok = true;
    if (model == 1) {
        stvk_eval(F, mu, lam, ps, P);
        stvk_hessian_projected<double>(F, mu, lam, M, W);
    } else if (model == 2) {
        ok = fcr_eval(F, mu, lam, ps, P);
        if (ok) fcr_hessian_projected<double>(F, mu, lam, M, W);
    } else {
        ok = nh_eval(F, mu, lam, ps, P, nullptr);
        if (ok) nh_hessian_projected<double>(F, mu, lam, M);
    }
    if (!ok) {
        psi[i] = INFINITY;
        return;
    }
    psi[i] = ps;
    for (int a = 0; a < 9; ++a) {
        g[9 * (size_t)i + a] = P[a];
        for (int b = 0; b < 9; ++b) H[81 * (size_t)i + 9 * a + b] = M(a, b);
    }
}

__global__ void k_local_accd(const double* x12, const double* p12, const int* is_ee, int n, double* t) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    V3 x[4], p[4];
    for (int k = 0; k < 4; ++k) {
        x[k] = ld3(x12 + 12 * (size_t)i + 3 * k);
        p[k] = ld3(p12 + 12 * (size_t)i + 3 * k);
    }
    t[i] = accd(x, p, is_ee[i] != 0, 0.1, 1.0, 10000, nullptr);
}

template <class T>
void get(T* h, const T* d, size_t n, cudaStream_t st) {
    if (n) ZCHECK(cudaMemcpyAsync(h, d, n * sizeof(T), cudaMemcpyDeviceToHost, st));
}

zema_status status_of(const ZemaError& e) { return (zema_status)e.status; }

}  // namespace

extern "C" {

zema_status zema_candidates_raw(int64_t nsv, const double* pos0, const double* pos1, const int32_t* sv_body, int64_t nb,
                                const int32_t* b_class, const int32_t* b_env, int64_t ne, const int32_t* edges,
                                int64_t nt, const int32_t* tris, double inflate, double cell_size, int64_t cap,
                                int32_t* pt_out, int32_t* ee_out, int64_t* n_out, void* stream) {
    set_current_stream((cudaStream_t)stream);
    if (nsv < 0 || nb < 1 || ne < 0 || nt < 0 || !pos0 || !sv_body || !b_class || !b_env || !n_out || !(inflate >= 0))
        return ZEMA_ERR_INVALID_ARG;
    try {
        cudaStream_t st = (cudaStream_t)stream;
        Temp T(st);
        double cs = cell_size;
        if (!(cs > 0)) {
            double sum = 0.0;
            for (int64_t i = 0; i < ne; ++i) {
                double d2 = 0.0;
                for (int j = 0; j < 3; ++j) {
                    double d = pos0[3 * edges[2 * i] + j] - pos0[3 * edges[2 * i + 1] + j];
                    d2 += d * d;
                }
                sum += std::sqrt(d2);
            }
            cs = std::max(ne ? sum / ne : 2.0 * inflate, 2.0 * inflate);
            if (!(cs > 0)) cs = 1.0;
        }
        BPView v;
        v.nsv = (int)nsv;
        v.ne = (int)ne;
        v.nt = (int)nt;
        v.X0 = T.put(pos0, 3 * (size_t)nsv);
        v.X1 = pos1 ? T.put(pos1, 3 * (size_t)nsv) : nullptr;
        int* svb = T.put(sv_body, (size_t)nsv);
        v.sv_body = svb;
        v.body_class = T.put(b_class, (size_t)nb);
        int* benv = T.put(b_env, (size_t)nb);
        int* sve = T.put<int>(nullptr, (size_t)nsv + 1);
        if (nsv) ZL(k_sv_env_of, div_up(nsv, TB), TB, 0, st)(svb, benv, (int)nsv, sve);
        ZLAUNCH();
        v.sv_env = sve;
        v.edges = (const int2*)T.put(edges, 2 * (size_t)ne);
        v.tris = (const int3*)T.put(tris, 3 * (size_t)nt);
        v.infl = inflate;
        v.inv_cell = 1.0 / cs;
        BroadPhase bp;
        bp.run(&T.A, v, st);
        n_out[0] = bp.n_pt;
        n_out[1] = bp.n_ee;
        std::vector<int2> h;
        if (pt_out) {
            size_t m = std::min<size_t>(bp.n_pt, (size_t)cap);
            h.resize(m);
            get(h.data(), bp.pt.p, m, st);
            ZCHECK(cudaStreamSynchronize(st));
            for (size_t i = 0; i < m; ++i) {
                pt_out[2 * i] = h[i].x;
                pt_out[2 * i + 1] = h[i].y;
            }
        }
        if (ee_out) {
            size_t m = std::min<size_t>(bp.n_ee, (size_t)cap);
            h.resize(m);
            get(h.data(), bp.ee.p, m, st);
            ZCHECK(cudaStreamSynchronize(st));
            for (size_t i = 0; i < m; ++i) {
                ee_out[2 * i] = h[i].x;
                ee_out[2 * i + 1] = h[i].y;
            }
        }
        ZCHECK(cudaStreamSynchronize(st));
        // release the broad phase's buffers before the temp allocator goes
        bp.~BroadPhase();
        new (&bp) BroadPhase();
        return ZEMA_OK;
    } catch (const ZemaError& e) {
        return status_of(e);
    }
}

zema_status zema_local_barrier(int64_t n, const double* x12, const int32_t* is_ee, const double* eps_x, double dhat,
                               double* e_out, double* g_out, double* H_out, void* stream) {
    set_current_stream((cudaStream_t)stream);
    if (n < 0 || !x12 || !is_ee || !eps_x || !e_out || !g_out || !H_out || !(dhat > 0)) return ZEMA_ERR_INVALID_ARG;
    if (n == 0) return ZEMA_OK;
    try {
        cudaStream_t st = (cudaStream_t)stream;
        Temp T(st);
        double* dx = T.put(x12, 12 * (size_t)n);
        int* de = T.put(is_ee, (size_t)n);
        double* dp = T.put(eps_x, (size_t)n);
        double* E = T.put<double>(nullptr, (size_t)n);
        double* g = T.put<double>(nullptr, 12 * (size_t)n);
        double* H = T.put<double>(nullptr, 144 * (size_t)n);
        int* flag = T.put<int>(nullptr, (size_t)n);
        ZL(k_local_barrier, div_up(n, kRawThreads), kRawThreads, 0, st)(dx, de, dp, (int)n, dhat, E, g, H, flag);
        ZL(k_local_project, div_up(n, kProjPairs), kCoopLanes * kProjPairs, 0, st)((int)n, flag, H);
        ZLAUNCH();
        get(e_out, E, n, st);
        get(g_out, g, 12 * n, st);
        get(H_out, H, 144 * n, st);
        ZCHECK(cudaStreamSynchronize(st));
        return ZEMA_OK;
    } catch (const ZemaError& e) {
        return status_of(e);
    }
}

zema_status zema_local_distance(int64_t n, const double* x12, const int32_t* is_ee, double* d2_out, double* w_out,
                                void* stream) {
    set_current_stream((cudaStream_t)stream);
    if (n < 0 || !x12 || !is_ee || !d2_out || !w_out) return ZEMA_ERR_INVALID_ARG;
    if (n == 0) return ZEMA_OK;
    try {
        cudaStream_t st = (cudaStream_t)stream;
        Temp T(st);
        double* dx = T.put(x12, 12 * (size_t)n);
        int* de = T.put(is_ee, (size_t)n);
        double* d2 = T.put<double>(nullptr, (size_t)n);
        double* w = T.put<double>(nullptr, 4 * (size_t)n);
        ZL(k_local_distance, div_up(n, 128), 128, 0, st)(dx, de, (int)n, d2, w);
        ZLAUNCH();
        get(d2_out, d2, n, st);
        get(w_out, w, 4 * n, st);
        ZCHECK(cudaStreamSynchronize(st));
        return ZEMA_OK;
    } catch (const ZemaError& e) {
        return status_of(e);
    }
}

zema_status zema_local_neo_hookean(int64_t n, const double* F9, double mu, double lam, double* psi_out, double* g_out,
                                   double* H_out, void* stream) {
    set_current_stream((cudaStream_t)stream);
    if (n < 0 || !F9 || !psi_out || !g_out || !H_out) return ZEMA_ERR_INVALID_ARG;
    if (n == 0) return ZEMA_OK;
    try {
        cudaStream_t st = (cudaStream_t)stream;
        Temp T(st);
        double* dF = T.put(F9, 9 * (size_t)n);
        double* ps = T.put<double>(nullptr, (size_t)n);
        double* g = T.put<double>(nullptr, 9 * (size_t)n);
        double* H = T.put<double>(nullptr, 81 * (size_t)n);
        ZCHECK(cudaFuncSetAttribute(k_local_nh, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 81 * EL_T * 8));
        ZL(k_local_nh, div_up(n, EL_T), EL_T, 2 * 81 * EL_T * 8, st)(dF, (int)n, mu, lam, ps, g, H);
        ZLAUNCH();
        get(psi_out, ps, n, st);
        get(g_out, g, 9 * n, st);
        get(H_out, H, 81 * n, st);
        ZCHECK(cudaStreamSynchronize(st));
        return ZEMA_OK;
    } catch (const ZemaError& e) {
        return status_of(e);
    }
}

zema_status zema_local_elastic(int64_t n, const double* F9, double mu, double lam, int32_t model, double* psi_out,
                               double* g_out, double* H_out, void* stream) {
    set_current_stream((cudaStream_t)stream);
    if (n < 0 || !F9 || !psi_out || !g_out || !H_out || model < 0 || model > 2) return ZEMA_ERR_INVALID_ARG;
    if (n == 0) return ZEMA_OK;
    try {
        cudaStream_t st = (cudaStream_t)stream;
        Temp T(st);
        double* dF = T.put(F9, 9 * (size_t)n);
        double* ps = T.put<double>(nullptr, (size_t)n);
        double* g = T.put<double>(nullptr, 9 * (size_t)n);
        double* H = T.put<double>(nullptr, 81 * (size_t)n);
        ZCHECK(cudaFuncSetAttribute(k_local_elastic, cudaFuncAttributeMaxDynamicSharedMemorySize, 81 * EL_T * 8));
        ZL(k_local_elastic, div_up(n, EL_T), EL_T, 81 * EL_T * 8, st)(dF, (int)n, mu, lam, model, ps, g, H);
        ZLAUNCH();
        get(psi_out, ps, n, st);
        get(g_out, g, 9 * n, st);
        get(H_out, H, 81 * n, st);
        ZCHECK(cudaStreamSynchronize(st));
        return ZEMA_OK;
    } catch (const ZemaError& e) {
        return status_of(e);
    }
}

zema_status zema_local_accd(int64_t n, const double* x12, const double* p12, const int32_t* is_ee, double* t_out,
                            void* stream) {
    set_current_stream((cudaStream_t)stream);
    if (n < 0 || !x12 || !p12 || !is_ee || !t_out) return ZEMA_ERR_INVALID_ARG;
    if (n == 0) return ZEMA_OK;
    try {
        cudaStream_t st = (cudaStream_t)stream;
        Temp T(st);
        double* dx = T.put(x12, 12 * (size_t)n);
        double* dp = T.put(p12, 12 * (size_t)n);
        int* de = T.put(is_ee, (size_t)n);
        double* t = T.put<double>(nullptr, (size_t)n);
        ZL(k_local_accd, div_up(n, 128), 128, 0, st)(dx, dp, de, (int)n, t);
        ZLAUNCH();
        get(t_out, t, n, st);
        ZCHECK(cudaStreamSynchronize(st));
        return ZEMA_OK;
    } catch (const ZemaError& e) {
        return status_of(e);
    }
}

}  // extern "C"
