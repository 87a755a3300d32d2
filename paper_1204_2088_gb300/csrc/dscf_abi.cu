// C ABI of the library (declared in include/dscf.h): parameter validation, the layout of the
// caller's workspace, replica tiling, capture of one time step into a CUDA graph, and the
// entry points.  Device memory is never allocated here.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/dscf.h"
#include "dscf_internal.cuh"

using namespace dscf;

namespace {

thread_local std::string g_init_error;

struct Layout {
    std::vector<Rep> reps;          // host copy, pointers filled by place()
    std::vector<int> tile2rep, blk2rep;
    std::vector<int> fwd_grid;      // [s] for s = 1..Nmax (index s), tiles of replicas with N >= s
    std::vector<size_t> fwd_smem, bwd_smem;   // [s] dynamic shared memory of the contour launches
    size_t es = 8;
    int ntiles = 0, nblk = 0, nlb = 0, Nmax = 0;
    bool w8 = false;                // every replica in whole rows of 256 sites
    size_t bytes = 0;
    // offsets of the shared blocks
    size_t off_reps = 0, off_t2r = 0, off_b2r = 0, off_status = 0;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool validate(const dscf_params* p, int n, std::string& why) {
    if (!p || n < 1) { why = "no replicas"; return false; }
    for (int r = 0; r < n; ++r) {
        const dscf_params& q = p[r];
        char buf[160];
        auto bad = [&](const char* m) { snprintf(buf, sizeof buf, "replica %d: %s", r, m); why = buf; return false; };
        if (q.nx < 1 || q.ny < 1 || q.nz < 1) return bad("grid sizes must be >= 1");
        if ((long long)q.nx * q.ny * q.nz > (1LL << 31) - 1) return bad("grid too large");
        if (q.ns != 2 && q.ns != 3) return bad("ns must be 2 or 3");
        if (q.N < 2 || q.N > 4096 || q.nA < 1 || q.nA >= q.N) return bad("need 1 <= nA < N <= 4096");
        if (!(q.phi_p > 0.0 && q.phi_p <= 1.0)) return bad("phi_p must be in (0, 1]");
        if (q.ns == 2 && q.phi_p != 1.0) return bad("a melt (ns = 2) needs phi_p = 1");
        const double al = q.a * q.a / 6.0;
        if (!(q.a > 0.0) || !(al < 0.5)) return bad("segment length must satisfy 0 < a^2/6 < 1/2");
        if (!(q.dt > 0.0) || !(q.M >= 0.0)) return bad("dt > 0 and M >= 0 required");
        if (!(q.tau_s > 0.5) || !(q.tau_b > 0.5)) return bad("LB relaxation times must exceed 1/2");
        if (!(q.rho0 > 0.0)) return bad("rho0 must be positive");
        if (q.ncg_iters < 0 || q.ncg_iters > kMaxNcg) return bad("ncg_iters must be in 0..32");
        if (q.cn_sweeps < 2 || q.cn_sweeps > 64 || (q.cn_sweeps & 1)) return bad("cn_sweeps must be even, 2..64");
        if (!(q.phi_floor > 0.0)) return bad("phi_floor must be positive");
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                if (q.chi[3 * i + j] != q.chi[3 * j + i] || (i == j && q.chi[3 * i + j] != 0.0))
                    return bad("chi must be symmetric with zero diagonal");
        if (q.ncg_iters != p[0].ncg_iters || q.cn_sweeps != p[0].cn_sweeps || q.hydro != p[0].hydro)
            return bad("ncg_iters, cn_sweeps and hydro must be the same for all replicas");
    }
    return true;
}

// Assign tiles (replicas in order of decreasing chain length own the first tiles, so the
// replicas still active at contour step s are a prefix) and per-step grid sizes, for the
// current z-chunk of every replica.
void assign_tiles(Layout& L, const dscf_params* p, int n) {
    // Flat kernels: about kMaxFlatBlocks blocks over the whole batch (one wave of four per SM).  A
    // replica whose own tiling would give it smaller chunks takes the batch's common chunk, so a
    // batch of many replicas does not launch tens of thousands of short blocks.  (A single
    // replica, or a batch of fewer than kMaxFlatBlocks x kFlatThreads sites, keeps its own tiling
    // and so its solo reduction order.)
    {
        long long Vtot = 0;
        for (int r = 0; r < n; ++r) Vtot += L.reps[r].V;
        long long common = (Vtot + kMaxFlatBlocks - 1) / kMaxFlatBlocks;
        common = (common + kFlatThreads - 1) / kFlatThreads * kFlatThreads;
        for (int r = 0; r < n; ++r) {
            Rep& R = L.reps[r];
            if (common > R.chunk) {
                R.chunk = (int)common;
                R.nblk = (int)((R.V + common - 1) / common);
            }
        }
    }
    std::vector<int> order(n);
    for (int r = 0; r < n; ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return p[a].N > p[b].N; });
    L.tile2rep.clear();
    L.blk2rep.clear();
    L.ntiles = 0;
    L.nblk = 0;
    L.nlb = 0;
    for (int r = 0; r < n; ++r) {
        L.reps[r].lb_blk0 = L.nlb;
        L.nlb += L.reps[r].lb_nblk;
    }
    for (int k = 0; k < n; ++k) {
        Rep& R = L.reps[order[k]];
        R.tile0 = L.ntiles;
        for (int t = 0; t < R.ntiles; ++t) L.tile2rep.push_back(order[k]);
        L.ntiles += R.ntiles;
        R.blk0 = L.nblk;
        for (int b = 0; b < R.nblk; ++b) L.blk2rep.push_back(order[k]);
        L.nblk += R.nblk;
    }
    L.fwd_grid.assign(L.Nmax + 2, 0);
    L.fwd_smem.assign(L.Nmax + 2, 0);
    L.bwd_smem.assign(L.Nmax + 2, 0);
    for (int s = 1; s <= L.Nmax; ++s)
        for (int r = 0; r < n; ++r)
            if (L.reps[r].N >= s) {
                L.fwd_grid[s] += L.reps[r].ntiles;
                L.fwd_smem[s] = std::max(L.fwd_smem[s], prop_smem_bytes(L.reps[r].vec, false, L.es));
                L.bwd_smem[s] = std::max(L.bwd_smem[s], prop_smem_bytes(L.reps[r].vec, true, L.es));
            }
}

int default_zc(int nz) { return std::min(nz, 8); }
constexpr int kPersSpinLimit = 1 << 22;   // polls (~64 ns sleep each) before a persistent sweep gives up

// Tiling and workspace layout.  With base == nullptr only sizes are computed.  Tile maps and
// partial-sum slots are sized for the smallest z-chunk the autotuner may choose, so re-tiling
// never moves anything.
Layout make_layout(const dscf_params* p, int n, int prec, char* base) {
    Layout L;
    const size_t es = (prec == DSCF_FP64) ? sizeof(double) : sizeof(float);
    L.es = es;
    L.reps.resize(n);
    long long ext = 0, vb = 0;
    int max_tiles_total = 0, max_blk_total = 0;
    L.w8 = true;
    for (int r = 0; r < n; ++r) L.w8 = L.w8 && p[r].nx == 256;
    for (int r = 0; r < n; ++r) {
        Rep& R = L.reps[r];
        std::memset(&R, 0, sizeof(Rep));
        R.rep_index = r;
        const dscf_params& q = p[r];
        R.nx = q.nx; R.ny = q.ny; R.nz = q.nz; R.ns = q.ns; R.N = q.N; R.nA = q.nA;
        R.V = (long long)q.nx * q.ny * q.nz;
        tile_replica(R, kMinZc, L.w8);
        const int max_tiles = R.ntiles;
        max_tiles_total += max_tiles;
        max_blk_total += R.nblk;
        R.part_stride = std::max(std::max(max_tiles, R.nblk), R.lb_nblk);
        tile_replica(R, default_zc(q.nz), L.w8);
        R.hydro = q.hydro;
        R.cn_sweeps = q.cn_sweeps;
        R.phi_p = q.phi_p; R.kappa = q.kappa; R.alpha = q.a * q.a / 6.0; R.dt = q.dt; R.M = q.M;
        R.gs = 1.0 - 1.0 / q.tau_s; R.gb = 1.0 - 1.0 / q.tau_b; R.rho0 = q.rho0; R.phi_floor = q.phi_floor;
        for (int i = 0; i < 9; ++i) R.chi[i] = q.chi[i];
        const double f = (double)q.nA / q.N;
        R.mass0[0] = (double)R.V * q.phi_p * f;
        R.mass0[1] = (double)R.V * q.phi_p * (1.0 - f);
        R.mass0[2] = q.ns == 3 ? (double)R.V * (1.0 - q.phi_p) : 0.0;
        R.ext_off = ext;
        R.vbase = vb;
        ext += (long long)q.ns * R.V;
        vb += R.V;
        L.Nmax = std::max(L.Nmax, q.N);
    }
    assign_tiles(L, p, n);
    // workspace
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        void* ptr = base ? (void*)(base + off) : nullptr;
        off = align256(off + bytes);
        return ptr;
    };
    for (int r = 0; r < n; ++r) {
        Rep& R = L.reps[r];
        const size_t V = (size_t)R.V, ns = (size_t)R.ns;
        R.phi = take(ns * V * es);
        R.U = take(ns * V * es);
        R.mu = take(ns * V * es);
        R.d = take(ns * V * es);
        R.phim = take(ns * V * es);
        R.q = take(2 * V * es);
        R.E = take(ns * V * es);
        R.G = take((size_t)R.N * V * es);
        R.Gp0 = take(V * es);
        R.Gp1 = take(V * es);
        R.u = take(3 * V * es);
        R.pop0 = take(19 * V * es);
        R.pop1 = take(19 * V * es);
        R.del0 = take(ns * V * es);
        R.del1 = take(ns * V * es);
        R.rhs = take(ns * V * es);
        R.Uprev = take(ns * V * es);
        R.part = (double*)take((size_t)NPART * R.part_stride * sizeof(double));
        R.scal = (double*)take((size_t)kScalStride * sizeof(double));
    }
    L.off_reps = off; take(sizeof(Rep) * n);
    L.off_t2r = off; take(sizeof(int) * max_tiles_total);
    L.off_b2r = off; take(sizeof(int) * max_blk_total);
    L.off_status = off; take(sizeof(int) * kStatusInts);
    L.bytes = off;
    return L;
}

__global__ void k_fill(double* p, long long n, double v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) p[i] = v;
}
__global__ void k_fillf(float* p, long long n, float v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) p[i] = v;
}

}  // namespace

namespace dscf {
// Message for dscf_last_error(NULL) from entry points that have no context.
void set_thread_error(const char* msg) { g_init_error = msg ? msg : ""; }
}  // namespace dscf

struct dscf_ctx {
    int nrep = 0, prec = 0, device = 0;
    std::vector<dscf_params> params;
    Layout L;
    char* ws = nullptr;
    cudaStream_t stream = nullptr, cap = nullptr, cap_body = nullptr;   // graph capture; conditional bodies
    Rep* d_reps = nullptr;
    int* d_t2r = nullptr;
    int* d_b2r = nullptr;
    int* d_status = nullptr;
    int* d_counter = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool probe = false, probe_ran = false;
    cudaEvent_t ev[6] = {};
    bool phim_stale = true;
    int zc = 0;
    // learned predictor (see dscf_set_predictor)
    dscf_net* net = nullptr;
    int pred_k = 10, pred_iters = 0;   // corrector period; inversion iterations of predictor steps
    double pred_tol = 1e-3;
    bool pred_ok = false, last_was_pred = false;
    long long pred_counter = 0, n_pred = 0, n_exact = 0;
    double pred_err = -1.0;
    cudaGraphExec_t exec_pred = nullptr;
    int kfuse = 1;          // contour steps per propagator launch (1 = single-step kernels, 0 = persistent)
    int pers_bz = 0;        // brick depth of the persistent sweeps (0 = not available)
    int pers_nw = 16;       // warps per CTA of the persistent sweeps
    struct PersGroup { int width, pby, first, nbricks; };   // one cooperative launch per sweep direction
    std::vector<PersGroup> pgroups;                    // brick table entries [first, first + nbricks)
    int wait_limit = kPersSpinLimit;   // polls before a persistent sweep gives up on a neighbour
    double ncg_tol = 0.0;   // > 0: residual stop of the inversion (conditional graph nodes)
    int warm = 0;           // 1: the inversion starts from the potentials extrapolated in time
    int noise = 0;          // thermal noise (dscf_set_noise): 1 compositions, 2 LB modes
    cudaError_t cap_err = cudaSuccess;   // first graph-construction error of a capture
    const char* cap_what = "";
    int nsm = 0;
    bool fusable = false;   // FP32 and every replica in the whole-row layout
    long long steps = 0;
    int64_t launches = 0;
    std::string err;
};

namespace {

int fail(dscf_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_init_error = buf;
    return code;
}

int cuda_check(dscf_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return DSCF_OK;
    return fail(c, DSCF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

Launch launch_of(dscf_ctx* c, cudaStream_t s) {
    Launch L;
    L.reps = c->d_reps;
    L.tile2rep = c->d_t2r;
    L.blk2rep = c->d_b2r;
    L.status = c->d_status;
    L.counter = c->d_counter;
    L.nblk_total = c->L.nblk;
    L.nlb_total = c->L.nlb;
    L.nrep = c->nrep;
    L.noise = c->noise;
    L.stream = s;
    L.w8 = c->L.w8 ? 1 : 0;
    return L;
}

// The persistent sweeps require equal step counters of all bricks at launch: re-arm them whenever
// the brick decomposition changes.
int reset_pers_flags(dscf_ctx* c) {
    return cuda_check(c, cudaMemsetAsync(c->d_status + kFlagBase, 0, sizeof(int) * (size_t)kMaxBricks * kFlagStride, c->stream),
                      "re-arming the brick counters");
}

int* pers_flags(dscf_ctx* c) { return c->d_status + kFlagBase; }
int4* pers_table(dscf_ctx* c) { return (int4*)(c->d_status + kFlagBase + (size_t)kMaxBricks * kFlagStride); }
int pers_total_bricks(const dscf_ctx* c) {
    int t = 0;
    for (const Rep& R : c->L.reps) t += pers_bricks(R, c->pers_bz);
    return t;
}

// Launch groups and brick table of the persistent sweeps.  The replicas are packed into
// cooperative launches of at most as many bricks as can be co-resident (one per SM for bricks of
// 16 planes, two for 8), every replica's bricks in one launch (they wait on one another): first
// fit, replicas taken by decreasing chain length and then decreasing brick count, so that a launch
// (which lasts as long as its longest chain) mostly holds chains of equal length.  A launch whose
// replicas share one row width and brick height runs that width's kernel, any other the
// mixed-width kernel (rows of 32 to 96 sites; 128-wide replicas share launches only with each
// other).  Each brick's step counter is at its replica's flag base (the replicas'
// bricks in index order).
// Placement: the CTAs of a sweep-shaped cooperative launch land on SMs in a fixed pattern that
// scatters consecutive CTA indices over the GPCs (and both dies); within a launch the bricks are
// given to the CTAs in the order of their SM ids instead, so that the bricks of one z slab
// (consecutive brick indices, y fastest) share a GPC and neighbouring slabs sit on neighbouring
// GPCs.  The table is a permutation: correctness does not depend on the placement repeating.
int place_bricks(dscf_ctx* c) {
    c->pgroups.clear();
    const int n = c->nrep, bz = c->pers_bz;
    const int cap = std::min(c->nsm * (c->pers_nw == 8 ? 2 : 1), kMaxBricks);
    std::vector<int> fbase(n), nbr(n), order(n);
    int tot = 0;
    for (int r = 0; r < n; ++r) {
        fbase[r] = tot;
        nbr[r] = pers_bricks(c->L.reps[r], bz);
        tot += nbr[r];
        order[r] = r;
        if (nbr[r] > cap)
            return fail(c, DSCF_ERR_ARG, "persistent sweeps: replica %d has %d bricks, more than %d", r, nbr[r], cap);
    }
    if (tot > kMaxBricks) return fail(c, DSCF_ERR_ARG, "persistent sweeps: %d bricks exceed %d", tot, kMaxBricks);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const Rep &A = c->L.reps[a], &B = c->L.reps[b];
        return A.N != B.N ? A.N > B.N : nbr[a] > nbr[b];
    });
    std::vector<std::vector<int>> bins;
    std::vector<int> load;
    auto wide = [&](int r) { return c->L.reps[r].nx == 128; };   // 128-wide replicas share launches only with each other
    for (int r : order) {
        size_t k = 0;
        while (k < bins.size() && (load[k] + nbr[r] > cap || wide(bins[k][0]) != wide(r))) ++k;
        if (k == bins.size()) { bins.emplace_back(); load.push_back(0); }
        bins[k].push_back(r);
        load[k] += nbr[r];
    }
    std::vector<int4> table(tot);
    int* d_smid = (int*)pers_table(c);   // probe scratch: the table is uploaded after the probes
    int first = 0;
    for (const auto& bin : bins) {
        std::vector<int4> ent;
        int width = c->L.reps[bin[0]].nx, pby = pers_pby(c->L.reps[bin[0]]);
        for (int r : bin) {
            const Rep& R = c->L.reps[r];
            if (R.nx != width || pers_pby(R) != pby) width = pby = 0;   // mixed widths
            for (int b = 0; b < nbr[r]; ++b) ent.push_back(make_int4(r, b, fbase[r], 0));
        }
        const int nb = (int)ent.size();
        std::vector<int> smid(nb), ord(nb);
        int rc = cuda_check(c, (cudaError_t)pers_placement(bz, c->pers_nw, nb, d_smid, c->stream), "placement probe");
        if (!rc) rc = cuda_check(c, cudaMemcpyAsync(smid.data(), d_smid, sizeof(int) * nb, cudaMemcpyDeviceToHost, c->stream),
                                 "placement probe");
        if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "placement probe");
        if (rc) { c->pgroups.clear(); return rc; }
        for (int i = 0; i < nb; ++i) ord[i] = i;
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return smid[a] < smid[b]; });
        for (int k = 0; k < nb; ++k) table[first + ord[k]] = ent[k];
        c->pgroups.push_back({width, pby, first, nb});
        first += nb;
    }
    int rc = cuda_check(c, cudaMemcpyAsync(pers_table(c), table.data(), sizeof(int4) * tot, cudaMemcpyHostToDevice, c->stream),
                        "brick table");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "brick table");
    if (rc) c->pgroups.clear();
    return rc;
}

// One direction of the persistent sweeps of every replica: one cooperative launch per group.
int64_t launch_pers_sweeps(dscf_ctx* c, const Launch& L, bool bwd, int limit) {
    for (const auto& g : c->pgroups)
        launch_prop_pers(L, bwd, g.width, g.pby, c->pers_bz, c->pers_nw, g.nbricks, pers_table(c) + g.first,
                         pers_flags(c), c->d_status + 2, limit);
    return (int64_t)c->pgroups.size();
}

// Forward and backward contour sweeps of one gradient evaluation.
template <typename T>
int64_t enqueue_sweeps(dscf_ctx* c, const Launch& L) {
    int64_t n = 0;
    const int K = c->kfuse;
    if (K == 0) {
        n += launch_pers_sweeps(c, L, false, c->wait_limit);
        n += launch_pers_sweeps(c, L, true, c->wait_limit);
        return n;
    }
    if (K > 1) {
        int vmax = 0;
        for (const Rep& R : c->L.reps) vmax = std::max(vmax, R.vec);
        const size_t sm = prop_fused_smem_bytes(vmax, K);
        const int ng = (c->L.Nmax + K - 1) / K;
        for (int g = 0; g < ng; ++g) { launch_prop_fused(L, false, K, g, c->L.fwd_grid[g * K + 1], sm); ++n; }
        for (int g = 0; g < ng; ++g) { launch_prop_fused(L, true, K, g, c->L.fwd_grid[g * K + 1], sm); ++n; }
        return n;
    }
    for (int s = 1; s <= c->L.Nmax; ++s) { launch_prop_fwd<T>(L, s, c->L.fwd_grid[s], c->L.fwd_smem[s]); ++n; }
    for (int j = 0; j < c->L.Nmax; ++j) { launch_prop_bwd<T>(L, j, c->L.fwd_grid[j + 1], c->L.bwd_smem[j + 1]); ++n; }
    return n;
}

// One gradient evaluation: Boltzmann factors, forward and backward contour sweeps.
template <typename T>
int64_t enqueue_eval(dscf_ctx* c, const Launch& L, int exp_mode, int k, const void* Uext) {
    int64_t n = 0;
    launch_exp<T>(L, exp_mode, k, Uext); ++n;
    n += enqueue_sweeps<T>(c, L);
    return n;
}

// The launch sequence of one time step (see include/dscf.h, steps 1-4).
// Learned-predictor evaluation at the potential the Boltzmann-factor kernel wrote into E:
// q <- phi_hat[U'] (FP32 melts, one replica).
void enqueue_net(dscf_ctx* c, const Launch& L) {
    const Rep& R = c->L.reps[0];
    const double f = (double)R.nA / R.N;
    dscf_net_forward_on(c->net, L.stream, (const float*)R.E, R.phi_p * f, R.phi_p * (1.0 - f), (float*)R.q);
}

// Conditional graph nodes for the residual stop of the inversion.  During a capture on c->cap,
// cond_begin appends an IF node on `h` after the captured work and starts capturing its body on
// c->cap_body; cond_end ends the body, and later work on c->cap follows the IF node.
cudaError_t cond_handle(dscf_ctx* c, cudaGraphConditionalHandle* h) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    c->cap_what = "capture info";
    cudaError_t e = cudaStreamGetCaptureInfo(c->cap, &st, nullptr, &g, nullptr, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    c->cap_what = "conditional handle";
    return cudaGraphConditionalHandleCreate(h, g, 0, cudaGraphCondAssignDefault);
}

cudaError_t cond_begin(dscf_ctx* c, cudaGraphConditionalHandle h) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    c->cap_what = "capture info (dependencies)";
    cudaError_t e = cudaStreamGetCaptureInfo(c->cap, &st, nullptr, &g, &deps, nullptr, &nd);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    c->cap_what = "add IF node";
    e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &np);
    if (e != cudaSuccess) return e;
    c->cap_what = "capture dependencies";
    e = cudaStreamUpdateCaptureDependencies(c->cap, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return e;
    c->cap_what = "begin body capture";
    return cudaStreamBeginCaptureToGraph(c->cap_body, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal);
}

cudaError_t cond_end(dscf_ctx* c) {
    c->cap_what = "launch in IF body";
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    c->cap_what = "end body capture";
    return cudaStreamEndCapture(c->cap_body, nullptr);
}

template <typename T>
int64_t enqueue_step(dscf_ctx* c, const Launch& L, bool pred = false) {
    const int K = pred ? c->pred_iters : c->params[0].ncg_iters;
    // residual stop: each exact iteration k sits in an IF node whose condition (a handle of its
    // own: a handle belongs to one conditional node) the gate kernel before it sets from the
    // residual the previous iteration left (a skipped iteration leaves it unchanged, so once
    // closed every later gate stays closed)
    const bool gate = !pred && K > 0 && c->ncg_tol > 0.0;
    auto mark = [&](int i) {
        if (c->probe && !pred && !(gate && i < 2)) cudaEventRecordWithFlags(c->ev[i], L.stream, cudaEventRecordExternal);
    };
    auto note = [&](cudaError_t e) {
        if (c->cap_err == cudaSuccess && e != cudaSuccess) c->cap_err = e;
    };
    int64_t n = 0;
    mark(4);
    if (!pred && c->warm && K > 0) {
        // start from 2 U^{n-1} - U^{n-2} (once two steps have produced potentials) and evaluate
        // phi there, the inversion's starting residual
        launch_extrap<T>(L); ++n;
        n += enqueue_eval<T>(c, L, 0, 0, nullptr);
        launch_grad<T>(L, -1); ++n;
    }
    if (K > 0) { launch_dir<T>(L, 0, 0); ++n; }
    for (int k = 0; k < K; ++k) {
        if (gate && c->cap_err == cudaSuccess) {
            cudaGraphConditionalHandle h = 0;
            note(cond_handle(c, &h));
            if (c->cap_err != cudaSuccess) break;
            launch_ncg_gate(L, k, c->ncg_tol, (unsigned long long)h); ++n;
            c->cap_what = "gate launch";
            note(cudaGetLastError());
            note(cond_begin(c, h));
            if (c->cap_err != cudaSuccess) break;
            const Launch Lb = launch_of(c, c->cap_body);
            launch_exp<T>(Lb, 1, k, nullptr); ++n;
            n += enqueue_sweeps<T>(c, Lb);
            launch_trial<T>(Lb); ++n;
            n += enqueue_eval<T>(c, Lb, 2, k, nullptr);
            launch_grad<T>(Lb, k); ++n;
            if (k + 1 < K) { launch_dir<T>(Lb, 1, k); ++n; }
            note(cond_end(c));
            continue;
        }
        if (pred) {   // both evaluations of the iteration through the learned predictor
            launch_exp<T>(L, 1, k, nullptr, 1); ++n;
            enqueue_net(c, L); n += dscf_net_forward_launches(c->net);
            launch_trial<T>(L, 1); ++n;
            launch_exp<T>(L, 2, k, nullptr, 1); ++n;
            enqueue_net(c, L); n += dscf_net_forward_launches(c->net);
            launch_grad<T>(L, k, 1); ++n;
            if (k + 1 < K) { launch_dir<T>(L, 1, k); ++n; }
            continue;
        }
        launch_exp<T>(L, 1, k, nullptr); ++n;
        if (k == 0) mark(0);
        n += enqueue_sweeps<T>(c, L);
        if (k == 0) mark(1);
        launch_trial<T>(L); ++n;
        n += enqueue_eval<T>(c, L, 2, k, nullptr);
        launch_grad<T>(L, k); ++n;
        if (k + 1 < K) { launch_dir<T>(L, 1, k); ++n; }
    }
    launch_mu<T>(L, gate ? -1 : K); ++n;
    if (c->params[0].hydro) {
        mark(2);
        launch_lb<T>(L, nullptr); ++n;
        mark(3);
        launch_step_end(L); ++n;
    } else if (c->noise) {
        launch_step_end(L); ++n;   // the step counter indexes the noise
    }
    launch_cd<T>(L, c->params[0].cn_sweeps);
    n += 3 + c->params[0].cn_sweeps;
    mark(5);
    return n;
}

// Forget the potentials' history (the extrapolated warm start restarts its count).
int reset_warm(dscf_ctx* c) {
    for (int r = 0; r < c->nrep; ++r) {
        const Rep& R = c->L.reps[r];
        if (int rc = cuda_check(c, cudaMemsetAsync(R.scal + S_WARM, 0, sizeof(double), c->stream), "warm-start reset"))
            return rc;
    }
    return DSCF_OK;
}

template <typename T>
int refresh_phim(dscf_ctx* c) {
    const Launch L = launch_of(c, c->stream);
    enqueue_eval<T>(c, L, 0, 0, nullptr);
    launch_grad<T>(L, -1);
    c->phim_stale = false;
    return cuda_check(c, cudaGetLastError(), "phi[U] refresh");
}

template <typename T>
int build_graph(dscf_ctx* c, bool pred = false) {
    cudaGraph_t g = nullptr;
    int rc = cuda_check(c, cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (rc) return rc;
    const Launch L = launch_of(c, c->cap);
    c->cap_err = cudaSuccess;
    const int64_t n = enqueue_step<T>(c, L, pred);
    if (!pred) c->launches = n;
    cudaError_t le = cudaGetLastError();
    cudaError_t ee = cudaStreamEndCapture(c->cap, &g);
    if (c->cap_err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        const std::string what = std::string("inversion residual stop: ") + c->cap_what;
        return cuda_check(c, c->cap_err, what.c_str());
    }
    if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_check(c, le, "kernel launch during capture"); }
    if (ee != cudaSuccess) return cuda_check(c, ee, "end capture");
    cudaError_t ie = cudaGraphInstantiate(pred ? &c->exec_pred : &c->exec, g, 0);
    cudaGraphDestroy(g);
    return cuda_check(c, ie, "graph instantiate");
}

// Judgement of the learned predictor at a corrector step (an exact step just run).
// After a predictor step the error is that step's self-consistency error ||phi[U] - phi*||_inf:
// the exact density at the potential the predictor-driven inversion produced against the
// composition it was inverted for, which the corrector's own inversion measures as its starting
// residual (it also holds the composition change of one step, ~1e-5).  Otherwise (first judgement,
// or after a fallback) the network's own error max |phi_hat[U] - phi[U]| at the exactly inverted
// potential stands in for it (the inversion error it causes is observed to be at most of that
// size).  A non-finite error fails.
int check_predictor(dscf_ctx* c, bool after_pred) {
    const Launch L = launch_of(c, c->stream);
    launch_exp<float>(L, 0, 0, nullptr, 1);
    enqueue_net(c, L);
    launch_pred_err(L);
    double s0[2] = {0.0, 0.0}, e = 0.0;
    const double* scal = c->L.reps[0].scal;
    int rc = cuda_check(c, cudaGetLastError(), "predictor check");
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(s0, scal + S_GG0, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                                c->stream), "inversion residual");
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(&e, scal + S_PERR, sizeof(double), cudaMemcpyDeviceToHost,
                                                c->stream), "predictor error");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "predictor sync");
    if (rc) return rc;
    if (after_pred) e = std::isfinite(s0[0]) ? s0[1] : INFINITY;
    c->pred_err = e;
    c->pred_ok = std::isfinite(e) && e <= c->pred_tol;
    return DSCF_OK;
}

int set_dev(dscf_ctx* c) { return cuda_check(c, cudaSetDevice(c->device), "cudaSetDevice"); }

int upload_tiles(dscf_ctx* c) {
    int rc = cuda_check(c, cudaMemcpyAsync(c->d_reps, c->L.reps.data(), sizeof(Rep) * c->nrep, cudaMemcpyHostToDevice,
                                           c->stream), "reps");
    if (rc) return rc;
    rc = cuda_check(c, cudaMemcpyAsync(c->d_t2r, c->L.tile2rep.data(), sizeof(int) * c->L.ntiles, cudaMemcpyHostToDevice,
                                       c->stream), "tile map");
    if (rc) return rc;
    rc = cuda_check(c, cudaMemcpyAsync(c->d_b2r, c->L.blk2rep.data(), sizeof(int) * c->L.nblk, cudaMemcpyHostToDevice,
                                       c->stream), "block map");
    if (rc) return rc;
    return cuda_check(c, cudaStreamSynchronize(c->stream), "tile upload");
}

void set_zc(dscf_ctx* c, int zc) {
    for (int r = 0; r < c->nrep; ++r) tile_replica(c->L.reps[r], std::min(zc, c->L.reps[r].nz), c->L.w8);
    assign_tiles(c->L, c->params.data(), c->nrep);
}

// Persistent-sweep candidates (one warp per plane of the brick): bricks of 16 planes (one CTA per
// SM) and bricks of 8 planes (two CTAs per SM).  The first becomes the context's persistent
// configuration.
bool pers_all_supported(const dscf_ctx* c, int bz, int nw) {
    if (c->prec != DSCF_FP32) return false;
    const int nsm = std::min(c->nsm, kMaxBricks / 2);
    long long tot = 0;
    for (const Rep& R : c->L.reps) {
        if (!pers_supported(R, bz, nw, nsm)) return false;
        tot += pers_bricks(R, bz);
    }
    return tot <= kMaxBricks;
}

int pers_select(dscf_ctx* c, std::vector<std::pair<int, int>>& pcand) {
    c->pers_bz = 0;
    pcand.clear();
    if (pers_all_supported(c, 16, 16)) pcand.push_back({16, 16});
    if (pers_all_supported(c, 8, 8)) pcand.push_back({8, 8});
    for (auto& pc : pcand) {
        for (const Rep& R : c->L.reps)
            if (int rc = cuda_check(c, (cudaError_t)pers_prepare(R.nx, pers_pby(R), pc.first, pc.second),
                                    "persistent sweep set-up"))
                return rc;
        if (int rc = cuda_check(c, (cudaError_t)pers_prepare(0, 0, pc.first, pc.second), "persistent sweep set-up"))
            return rc;
    }
    if (!pcand.empty()) {
        c->pers_bz = pcand[0].first;
        c->pers_nw = pcand[0].second;
    }
    return DSCF_OK;
}

// Fusion support and its shared-memory limit (needed before any fused launch).
int fusion_setup(dscf_ctx* c) {
    c->fusable = (c->prec == DSCF_FP32);
    for (const Rep& R : c->L.reps) c->fusable = c->fusable && (R.vec > 0);
    if (c->fusable) {
        const size_t lim = prop_fused_smem_bytes(4, 4);
        return cuda_check(c, (cudaError_t)prop_fused_set_smem_limit(lim), "fused shared-memory limit");
    }
    return DSCF_OK;
}

// Autotuner: pick the z-chunk of the propagator tiles and the number of contour steps fused per
// launch (one pair for all replicas) by timing forward contour launches on the context's own
// buffers; the figure of merit is time per contour step.  Small problems keep the defaults.
int autotune_zc(dscf_ctx* c) {
    long long Vtot = 0;
    int Nmin = 1 << 30;
    for (const Rep& R : c->L.reps) { Vtot += R.V; Nmin = std::min(Nmin, R.N); }
    int best = default_zc(c->L.reps[0].nz), bestK = 1;
    if (int rc = fusion_setup(c)) return rc;
    if (Vtot >= 32 * 32 * 32) {
        cudaEvent_t e0, e1;
        if (int rc = cuda_check(c, cudaEventCreate(&e0), "tune event")) return rc;
        if (int rc = cuda_check(c, cudaEventCreate(&e1), "tune event")) { cudaEventDestroy(e0); return rc; }
        float best_ms = 1e30f;
        const int cands[] = {4, 5, 6, 8, 11, 16, 22, 32};
        const int kmax = c->fusable ? std::min(c->L.w8 ? 2 : 4, Nmin) : 1;   // rows of 256 sites: two steps
        for (int zc : cands) {
            set_zc(c, zc);
            if (int rc = upload_tiles(c)) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
            const Launch L = launch_of(c, c->stream);
            for (int K = 1; K <= kmax; ++K) {
                int vmax = 0;
                for (const Rep& R : c->L.reps) vmax = std::max(vmax, R.vec);
                auto run = [&]() {
                    if (K == 1) {
                        if (c->prec == DSCF_FP64) launch_prop_fwd<double>(L, 2, c->L.fwd_grid[2], c->L.fwd_smem[2]);
                        else launch_prop_fwd<float>(L, 2, c->L.fwd_grid[2], c->L.fwd_smem[2]);
                    } else {
                        launch_prop_fused(L, false, K, 0, c->L.fwd_grid[1], prop_fused_smem_bytes(vmax, K));
                    }
                };
                for (int i = 0; i < 3; ++i) run();
                cudaEventRecord(e0, c->stream);
                for (int i = 0; i < 8; ++i) run();
                cudaEventRecord(e1, c->stream);
                float ms = 0.f;
                cudaError_t e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e == cudaSuccess) e = cudaGetLastError();
                if (e != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return cuda_check(c, e, "tune timing"); }
                ms /= (float)K;
                if (ms < best_ms) { best_ms = ms; best = zc; bestK = K; }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    // persistent sweeps (FP32, supported row widths; both brick depths): a forward and a backward
    // sweep of the whole batch per candidate, per sweep against the best above
    std::vector<std::pair<int, int>> pcand;
    if (int rc = pers_select(c, pcand)) return rc;
    if (!pcand.empty()) {
        c->pers_bz = pcand[0].first;
        c->pers_nw = pcand[0].second;
        if (Vtot >= 32 * 32 * 32 && Nmin >= 2) {
            // per contour step of the best multi-launch configuration, measured on a forward sweep
            auto sweep_ms = [&](int K, int zc) -> float {
                c->kfuse = K;
                set_zc(c, K == 0 ? c->pers_bz : zc);
                if (upload_tiles(c)) return 1e30f;
                const Launch L = launch_of(c, c->stream);
                cudaEvent_t e0, e1;
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                auto run = [&]() {
                    if (K == 0) {
                        launch_pers_sweeps(c, L, false, kPersSpinLimit);
                        launch_pers_sweeps(c, L, true, kPersSpinLimit);
                    } else if (c->prec == DSCF_FP64) {
                        enqueue_sweeps<double>(c, L);
                    } else {
                        enqueue_sweeps<float>(c, L);
                    }
                };
                run();
                cudaEventRecord(e0, c->stream);
                run();
                run();
                cudaEventRecord(e1, c->stream);
                float ms = 1e30f;
                if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                if (cudaGetLastError() != cudaSuccess) return 1e30f;
                return ms / 2.0f / 2.0f;   // per sweep, forward and backward
            };
            float tp = 1e30f;
            std::pair<int, int> pbest = pcand[0];
            for (auto& pc : pcand) {   // the first candidate (bricks of 16 planes) unless another is 2% faster
                c->pers_bz = pc.first;
                c->pers_nw = pc.second;
                if (int rc = reset_pers_flags(c)) return rc;
                if (int rc = place_bricks(c)) return rc;
                const float t = sweep_ms(0, 0);
                if (t < (tp < 1e29f ? 0.98f * tp : tp)) { tp = t; pbest = pc; }
            }
            c->pers_bz = pbest.first;
            c->pers_nw = pbest.second;
            if (int rc = reset_pers_flags(c)) return rc;
            if (int rc = place_bricks(c)) return rc;
            const float tm = sweep_ms(bestK, best);
            int st = 0;
            cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost);
            if (st & ST_TIMEOUT) return fail(c, DSCF_ERR_TIMEOUT, "persistent sweep timed out during tuning");
            if (tp < tm) bestK = 0;
        }
    }
    c->zc = bestK == 0 ? c->pers_bz : best;   // with persistent sweeps the brick depth
    c->kfuse = bestK;
    set_zc(c, bestK == 0 ? c->pers_bz : best);
    return upload_tiles(c);
}
// A tuning chosen earlier (for instance cached from an autotuner run) instead of the autotuner.
int apply_tuning(dscf_ctx* c, int zc, int kfuse) {
    std::vector<std::pair<int, int>> pcand;
    if (int rc = pers_select(c, pcand)) return rc;
    if (int rc = fusion_setup(c)) return rc;
    if (int rc = dscf_set_tuning(c, zc, kfuse)) return rc;
    if (kfuse == 0) {
        if (int rc = reset_pers_flags(c)) return rc;
        if (int rc = place_bricks(c)) return rc;
    }
    return DSCF_OK;
}
}  // namespace

extern "C" {

size_t dscf_workspace_bytes(const dscf_params* p, int32_t n, int32_t precision) {
    std::string why;
    if (precision != DSCF_FP64 && precision != DSCF_FP32) return 0;
    if (!validate(p, n, why)) return 0;
    return make_layout(p, n, precision, nullptr).bytes;
}

int dscf_init(const dscf_params* p, int32_t n, int32_t precision, void* workspace, size_t wbytes, void* stream,
              dscf_ctx** out) {
    return dscf_init_tuned(p, n, precision, workspace, wbytes, stream, -1, -1, out);
}

int dscf_init_tuned(const dscf_params* p, int32_t n, int32_t precision, void* workspace, size_t wbytes, void* stream,
                    int32_t zc, int32_t kfuse, dscf_ctx** out) {
    if (!out) return fail(nullptr, DSCF_ERR_ARG, "out is NULL");
    *out = nullptr;
    std::string why;
    if (precision != DSCF_FP64 && precision != DSCF_FP32) return fail(nullptr, DSCF_ERR_ARG, "bad precision");
    if (!validate(p, n, why)) return fail(nullptr, DSCF_ERR_ARG, "%s", why.c_str());
    if (!workspace || ((uintptr_t)workspace & 255)) return fail(nullptr, DSCF_ERR_ARG, "workspace must be 256-byte aligned");
    dscf_ctx* c = new (std::nothrow) dscf_ctx;
    if (!c) return fail(nullptr, DSCF_ERR_OOM, "host allocation failed");
    c->nrep = n;
    c->prec = precision;
    c->params.assign(p, p + n);
    c->stream = (cudaStream_t)stream;
    c->ws = (char*)workspace;
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, workspace) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        delete c;
        return fail(nullptr, DSCF_ERR_ARG, "workspace is not device memory");
    }
    c->device = pa.device;
    if (int rc = set_dev(c)) { g_init_error = c->err; delete c; return rc; }
    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
    c->L = make_layout(p, n, precision, c->ws);
    if (wbytes < c->L.bytes) {
        delete c;
        return fail(nullptr, DSCF_ERR_OOM, "workspace has %zu bytes, needs %zu", wbytes, c->L.bytes);
    }
    c->d_reps = (Rep*)(c->ws + c->L.off_reps);
    c->d_t2r = (int*)(c->ws + c->L.off_t2r);
    c->d_b2r = (int*)(c->ws + c->L.off_b2r);
    c->d_status = (int*)(c->ws + c->L.off_status);
    c->d_counter = c->d_status + 1;
    auto chk = [&](cudaError_t e, const char* w) { return cuda_check(c, e, w); };
    int rc = 0;
    rc = rc ? rc : chk(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking), "capture stream");
    rc = rc ? rc : chk(cudaStreamCreateWithFlags(&c->cap_body, cudaStreamNonBlocking), "capture stream");
    rc = rc ? rc : chk(cudaMemcpyAsync(c->d_reps, c->L.reps.data(), sizeof(Rep) * n, cudaMemcpyHostToDevice, c->stream), "reps");
    rc = rc ? rc : chk(cudaMemcpyAsync(c->d_t2r, c->L.tile2rep.data(), sizeof(int) * c->L.ntiles, cudaMemcpyHostToDevice, c->stream), "t2r");
    rc = rc ? rc : chk(cudaMemcpyAsync(c->d_b2r, c->L.blk2rep.data(), sizeof(int) * c->L.nblk, cudaMemcpyHostToDevice, c->stream), "b2r");
    rc = rc ? rc : chk(cudaMemsetAsync(c->d_status, 0, sizeof(int) * kStatusInts, c->stream), "status");
    const size_t es = precision == DSCF_FP64 ? 8 : 4;
    for (int r = 0; r < n && !rc; ++r) {
        const Rep& R = c->L.reps[r];
        const size_t V = (size_t)R.V;
        rc = rc ? rc : chk(cudaMemsetAsync(R.U, 0, R.ns * V * es, c->stream), "U");
        rc = rc ? rc : chk(cudaMemsetAsync(R.d, 0, R.ns * V * es, c->stream), "d");
        rc = rc ? rc : chk(cudaMemsetAsync(R.mu, 0, R.ns * V * es, c->stream), "mu");
        rc = rc ? rc : chk(cudaMemsetAsync(R.u, 0, 3 * V * es, c->stream), "u");
        rc = rc ? rc : chk(cudaMemsetAsync(R.pop0, 0, 19 * V * es, c->stream), "pop0");
        rc = rc ? rc : chk(cudaMemsetAsync(R.pop1, 0, 19 * V * es, c->stream), "pop1");
        rc = rc ? rc : chk(cudaMemsetAsync(R.part, 0, (size_t)NPART * R.part_stride * 8, c->stream), "part");
        rc = rc ? rc : chk(cudaMemsetAsync(R.scal, 0, (size_t)kScalStride * 8, c->stream), "scal");
        const double f = (double)R.nA / R.N;
        const double vals[3] = {R.phi_p * f, R.phi_p * (1.0 - f), 1.0 - R.phi_p};
        for (int I = 0; I < R.ns; ++I) {
            if (precision == DSCF_FP64)
                k_fill<<<256, 256, 0, c->stream>>>((double*)R.phi + I * V, (long long)V, vals[I]);
            else
                k_fillf<<<256, 256, 0, c->stream>>>((float*)R.phi + I * V, (long long)V, (float)vals[I]);
        }
    }
    rc = rc ? rc : chk(cudaGetLastError(), "fill");
    rc = rc ? rc : chk(cudaStreamSynchronize(c->stream), "init sync");
    if (!rc) {
        const size_t lim = std::max(prop_smem_bytes(4, true, c->L.es), prop_smem_bytes(0, true, c->L.es));
        const int e = precision == DSCF_FP64 ? prop_set_smem_limit<double>(lim) : prop_set_smem_limit<float>(lim);
        rc = cuda_check(c, (cudaError_t)e, "propagator shared-memory limit");
    }
    if (!rc) rc = (zc < 0) ? autotune_zc(c) : apply_tuning(c, zc, kfuse);
    if (rc) {
        g_init_error = c->err;
        if (c->cap) cudaStreamDestroy(c->cap);
        if (c->cap_body) cudaStreamDestroy(c->cap_body);
        delete c;
        return rc;
    }
    *out = c;
    return DSCF_OK;
}

int dscf_step(dscf_ctx* c, int32_t n_steps) {
    if (!c) return DSCF_ERR_ARG;
    if (n_steps < 0) return fail(c, DSCF_ERR_ARG, "n_steps < 0");
    if (int rc = set_dev(c)) return rc;
    if (c->phim_stale) {
        int rc = c->prec == DSCF_FP64 ? refresh_phim<double>(c) : refresh_phim<float>(c);
        if (rc) return rc;
    }
    if (!c->exec) {
        int rc = c->prec == DSCF_FP64 ? build_graph<double>(c) : build_graph<float>(c);
        if (rc) return rc;
    }
    if (!c->net) {
        for (int i = 0; i < n_steps; ++i) {
            if (int rc = cuda_check(c, cudaGraphLaunch(c->exec, c->stream), "graph launch")) return rc;
        }
        c->steps += n_steps;
        if (n_steps > 0 && c->probe) c->probe_ran = true;
        return DSCF_OK;
    }
    // learned predictor: every pred_k-th step is exact and judges the predictor; in between the
    // predictor is used while its last judgement was within tolerance, else the step is exact
    if (!c->exec_pred) {
        if (int rc = build_graph<float>(c, true)) return rc;
    }
    for (int i = 0; i < n_steps; ++i) {
        const bool check = (c->pred_counter % c->pred_k) == 0;
        const bool use_pred = !check && c->pred_ok;
        if (use_pred) {
            if (int rc = cuda_check(c, cudaGraphLaunch(c->exec_pred, c->stream), "predictor graph launch")) return rc;
            c->last_was_pred = true;
            ++c->n_pred;
        } else {
            const bool after_pred = c->last_was_pred;
            if (after_pred) {   // the exact inversion starts from the exact phi[U]
                if (int rc = refresh_phim<float>(c)) return rc;
            }
            if (int rc = cuda_check(c, cudaGraphLaunch(c->exec, c->stream), "graph launch")) return rc;
            c->last_was_pred = false;
            ++c->n_exact;
            if (check) {
                if (int rc = check_predictor(c, after_pred)) return rc;
            }
        }
        ++c->pred_counter;
        ++c->steps;
    }
    if (n_steps > 0 && c->probe) c->probe_ran = true;
    return DSCF_OK;
}

int dscf_densities(dscf_ctx* c, const void* U_in, void* phi_out) {
    if (!c || !U_in || !phi_out) return c ? fail(c, DSCF_ERR_ARG, "NULL field pointer") : DSCF_ERR_ARG;
    if (int rc = set_dev(c)) return rc;
    const Launch L = launch_of(c, c->stream);
    if (c->prec == DSCF_FP64) {
        enqueue_eval<double>(c, L, 3, 0, U_in);
        launch_dens_out<double>(L, phi_out);
    } else {
        enqueue_eval<float>(c, L, 3, 0, U_in);
        launch_dens_out<float>(L, phi_out);
    }
    // the propagator buffers no longer hold phi[U] of the context's U
    c->phim_stale = true;
    return cuda_check(c, cudaGetLastError(), "densities");
}

int lb_step(dscf_ctx* c, const void* force, int32_t n_steps) {
    if (!c) return DSCF_ERR_ARG;
    if (n_steps < 0) return fail(c, DSCF_ERR_ARG, "n_steps < 0");
    if (int rc = set_dev(c)) return rc;
    const Launch L = launch_of(c, c->stream);
    for (int i = 0; i < n_steps; ++i) {
        if (c->prec == DSCF_FP64) launch_lb<double>(L, force); else launch_lb<float>(L, force);
        launch_step_end(L);
    }
    return cuda_check(c, cudaGetLastError(), "lb_step");
}

int dscf_get_fields(dscf_ctx* c, int32_t which, void* dst, int32_t on_host) {
    if (!c || !dst) return c ? fail(c, DSCF_ERR_ARG, "NULL destination") : DSCF_ERR_ARG;
    if (int rc = set_dev(c)) return rc;
    const size_t es = c->prec == DSCF_FP64 ? 8 : 4;
    const cudaMemcpyKind kind = on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (which == DSCF_FIELD_POP) {
        if (on_host) return fail(c, DSCF_ERR_ARG, "populations are exchanged in device memory only");
        const Launch L = launch_of(c, c->stream);
        if (c->prec == DSCF_FP64) launch_pop_copy<double>(L, dst, 0); else launch_pop_copy<float>(L, dst, 0);
        return cuda_check(c, cudaGetLastError(), "get populations");
    }
    char* out = (char*)dst;
    for (int r = 0; r < c->nrep; ++r) {
        const Rep& R = c->L.reps[r];
        const size_t V = (size_t)R.V;
        const void* srcp = nullptr;
        size_t n = 0, off = 0;
        switch (which) {
            case DSCF_FIELD_PHI: srcp = R.phi; n = R.ns * V; off = R.ext_off; break;
            case DSCF_FIELD_U: srcp = R.U; n = R.ns * V; off = R.ext_off; break;
            case DSCF_FIELD_MU: srcp = R.mu; n = R.ns * V; off = R.ext_off; break;
            case DSCF_FIELD_PHIM: srcp = R.phim; n = R.ns * V; off = R.ext_off; break;
            case DSCF_FIELD_VEL: srcp = R.u; n = 3 * V; off = 3 * R.vbase; break;
            default: return fail(c, DSCF_ERR_ARG, "unknown field %d", which);
        }
        if (int rc = cuda_check(c, cudaMemcpyAsync(out + off * es, srcp, n * es, kind, c->stream), "get field")) return rc;
    }
    if (on_host) return cuda_check(c, cudaStreamSynchronize(c->stream), "get field sync");
    return DSCF_OK;
}

int dscf_set_fields(dscf_ctx* c, int32_t which, const void* src, int32_t on_host) {
    if (!c || !src) return c ? fail(c, DSCF_ERR_ARG, "NULL source") : DSCF_ERR_ARG;
    if (int rc = set_dev(c)) return rc;
    const size_t es = c->prec == DSCF_FP64 ? 8 : 4;
    const cudaMemcpyKind kind = on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const Launch L = launch_of(c, c->stream);
    if (which == DSCF_FIELD_POP) {
        if (on_host) return fail(c, DSCF_ERR_ARG, "populations are exchanged in device memory only");
        if (c->prec == DSCF_FP64) launch_pop_copy<double>(L, (void*)src, 1); else launch_pop_copy<float>(L, (void*)src, 1);
        return cuda_check(c, cudaGetLastError(), "set populations");
    }
    if (which != DSCF_FIELD_PHI && which != DSCF_FIELD_U) return fail(c, DSCF_ERR_ARG, "field %d cannot be set", which);
    const char* in = (const char*)src;
    for (int r = 0; r < c->nrep; ++r) {
        const Rep& R = c->L.reps[r];
        void* dstp = which == DSCF_FIELD_PHI ? R.phi : R.U;
        if (int rc = cuda_check(c, cudaMemcpyAsync(dstp, in + (size_t)R.ext_off * es, (size_t)R.ns * R.V * es, kind, c->stream),
                                "set field"))
            return rc;
    }
    if (which == DSCF_FIELD_PHI) {
        if (c->prec == DSCF_FP64) launch_mass_init<double>(L, c->nrep); else launch_mass_init<float>(L, c->nrep);
    } else {
        c->phim_stale = true;
    }
    if (int rc = reset_warm(c)) return rc;   // the history of the potentials no longer applies
    return cuda_check(c, cudaGetLastError(), "set field");
}

int dscf_observables(dscf_ctx* c, int32_t replica, double* out) {
    if (!c || !out) return c ? fail(c, DSCF_ERR_ARG, "NULL output") : DSCF_ERR_ARG;
    if (replica < 0 || replica >= c->nrep) return fail(c, DSCF_ERR_ARG, "replica out of range");
    if (int rc = set_dev(c)) return rc;
    // exact densities at the current potentials: Q (and the solvent sum) of Eq. 2
    int rc = c->prec == DSCF_FP64 ? refresh_phim<double>(c) : refresh_phim<float>(c);
    if (rc) return rc;
    const Launch L = launch_of(c, c->stream);
    const Rep& R = c->L.reps[replica];
    const int nb = R.nblk;
    std::vector<double> h((size_t)5 * nb);
    double qq[2] = {0.0, 0.0};
    if (c->prec == DSCF_FP64) launch_obs1<double>(L); else launch_obs1<float>(L);
    for (int k = 0; k < 5 && !rc; ++k)
        rc = cuda_check(c, cudaMemcpyAsync(h.data() + (size_t)k * nb, R.part + (size_t)(P_OBS0 + k) * R.part_stride,
                                           sizeof(double) * nb, cudaMemcpyDeviceToHost, c->stream), "observables");
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(qq, R.scal + S_Q, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                             "observables");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "observables sync");
    if (rc) return rc;
    double sum[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < 5; ++k)
        for (int i = 0; i < nb; ++i) sum[k] += h[(size_t)k * nb + i];   // fixed order
    const double V = (double)R.V;
    const double m[3] = {sum[0] / V, sum[1] / V, sum[2] / V};
    if (c->prec == DSCF_FP64) launch_obs2<double>(L, m[0], m[1], m[2]); else launch_obs2<float>(L, m[0], m[1], m[2]);
    for (int k = 0; k < 2 && !rc; ++k)
        rc = cuda_check(c, cudaMemcpyAsync(h.data() + (size_t)k * nb, R.part + (size_t)(P_OBS0 + k) * R.part_stride,
                                           sizeof(double) * nb, cudaMemcpyDeviceToHost, c->stream), "observables");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "observables sync");
    if (rc) return rc;
    double s2 = 0.0, seg = 0.0;
    for (int i = 0; i < nb; ++i) {
        s2 += h[i];
        seg += h[(size_t)nb + i];
    }
    const dscf_params& p = c->params[replica];
    double F = -p.phi_p / (double)p.N * std::log(qq[0]);
    if (p.ns == 3) F -= (1.0 - p.phi_p) * std::log(qq[1]);
    F += (-sum[3] + sum[4]) / V;
    out[0] = F;
    out[1] = std::sqrt(s2 / V);
    out[2] = seg / V;
    return DSCF_OK;
}

int dscf_minkowski(dscf_ctx* c, int32_t replica, int32_t species, double threshold, int64_t* counts) {
    if (!c || !counts) return c ? fail(c, DSCF_ERR_ARG, "NULL output") : DSCF_ERR_ARG;
    if (replica < 0 || replica >= c->nrep) return fail(c, DSCF_ERR_ARG, "replica out of range");
    const Rep& R = c->L.reps[replica];
    if (species < 0 || species >= R.ns) return fail(c, DSCF_ERR_ARG, "species out of range");
    if (!std::isfinite(threshold)) return fail(c, DSCF_ERR_ARG, "threshold must be finite");
    if (int rc = set_dev(c)) return rc;
    const Launch L = launch_of(c, c->stream);
    if (c->prec == DSCF_FP64) launch_minkowski<double>(L, replica, species, threshold);
    else launch_minkowski<float>(L, replica, species, threshold);
    const int nb = R.nblk;
    std::vector<double> h((size_t)4 * nb);
    int rc = cuda_check(c, cudaGetLastError(), "minkowski");
    for (int k = 0; k < 4 && !rc; ++k)
        rc = cuda_check(c, cudaMemcpyAsync(h.data() + (size_t)k * nb, R.part + (size_t)(P_OBS0 + k) * R.part_stride,
                                           sizeof(double) * nb, cudaMemcpyDeviceToHost, c->stream), "minkowski");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "minkowski sync");
    if (rc) return rc;
    for (int k = 0; k < 4; ++k) {
        long long s = 0;
        for (int b = 0; b < nb; ++b) s += (long long)h[(size_t)k * nb + b];
        counts[k] = s;
    }
    return DSCF_OK;
}

int dscf_trapped_solvent(dscf_ctx* c, int32_t replica, double threshold, double* out) {
    if (!c || !out) return c ? fail(c, DSCF_ERR_ARG, "NULL output") : DSCF_ERR_ARG;
    if (replica < 0 || replica >= c->nrep) return fail(c, DSCF_ERR_ARG, "replica out of range");
    const Rep& R = c->L.reps[replica];
    if (R.ns != 3) return fail(c, DSCF_ERR_ARG, "the replica has no solvent");
    if (!std::isfinite(threshold)) return fail(c, DSCF_ERR_ARG, "threshold must be finite");
    if (int rc = set_dev(c)) return rc;
    const Launch L = launch_of(c, c->stream);
    // scratch: the contour stack (recomputed by every density evaluation; N >= 2 levels of at least
    // 4 bytes per site) holds the 2 V ints of labels and counts
    int* lab = (int*)R.G;
    int* cnt = lab + R.V;
    int* changed = c->d_status + 3;
    if (c->prec == DSCF_FP64) launch_cc_init<double>(L, replica, threshold, lab, cnt);
    else launch_cc_init<float>(L, replica, threshold, lab, cnt);
    int rc = cuda_check(c, cudaGetLastError(), "trapped solvent");
    // label propagation to the fixed point, checked every 8 sweeps; bounded
    const long long max_sweeps = 64LL * ((long long)R.nx + R.ny + R.nz) + 1024;
    long long sweeps = 0;
    int ch = 1;
    while (!rc && ch) {
        if (sweeps > max_sweeps) return fail(c, DSCF_ERR_NOCONVERGE, "component labelling did not settle");
        rc = cuda_check(c, cudaMemsetAsync(changed, 0, sizeof(int), c->stream), "trapped solvent");
        for (int k = 0; k < 8 && !rc; ++k) launch_cc_step(L, replica, lab, changed);
        sweeps += 8;
        if (!rc) rc = cuda_check(c, cudaMemcpyAsync(&ch, changed, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                                 "trapped solvent");
        if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "trapped solvent");
    }
    if (rc) return rc;
    launch_cc_count(L, replica, lab, cnt);
    const int nb = R.nblk;
    std::vector<double> h((size_t)3 * nb);
    const int sl[3] = {P_OBS0, P_OBS1, P_OBS4};
    for (int k = 0; k < 3 && !rc; ++k)
        rc = cuda_check(c, cudaMemcpyAsync(h.data() + (size_t)k * nb, R.part + (size_t)sl[k] * R.part_stride,
                                           sizeof(double) * nb, cudaMemcpyDeviceToHost, c->stream), "trapped solvent");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "trapped solvent");
    if (rc) return rc;
    double bsize = -1.0, broot = -1.0, ncomp = 0.0;
    for (int b = 0; b < nb; ++b) {
        const double sz = h[b], rt = h[(size_t)nb + b];
        if (sz > bsize || (sz == bsize && rt < broot)) { bsize = sz; broot = rt; }
        ncomp += h[(size_t)2 * nb + b];
    }
    if (c->prec == DSCF_FP64) launch_cc_solvent<double>(L, replica, lab, (int)broot);
    else launch_cc_solvent<float>(L, replica, lab, (int)broot);
    for (int k = 0; k < 2 && !rc; ++k)
        rc = cuda_check(c, cudaMemcpyAsync(h.data() + (size_t)k * nb, R.part + (size_t)(P_OBS2 + k) * R.part_stride,
                                           sizeof(double) * nb, cudaMemcpyDeviceToHost, c->stream), "trapped solvent");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "trapped solvent");
    if (rc) return rc;
    double tr = 0.0, tot = 0.0;
    for (int b = 0; b < nb; ++b) {
        tr += h[b];
        tot += h[(size_t)nb + b];
    }
    out[0] = tot > 0.0 ? tr / tot : 0.0;
    out[1] = ncomp;
    return DSCF_OK;
}

int dscf_diagnostics(dscf_ctx* c, int32_t replica, double* out) {
    if (!c || !out || replica < 0 || replica >= c->nrep) return c ? fail(c, DSCF_ERR_ARG, "bad replica") : DSCF_ERR_ARG;
    if (int rc = set_dev(c)) return rc;
    double s[kScalStride];
    const Rep& R = c->L.reps[replica];
    {
        const Launch L = launch_of(c, c->stream);
        if (c->prec == DSCF_FP64) launch_lb_diag<double>(L); else launch_lb_diag<float>(L);
        if (int rc = cuda_check(c, cudaGetLastError(), "LB diagnostics")) return rc;
    }
    if (int rc = cuda_check(c, cudaMemcpyAsync(s, R.scal, sizeof s, cudaMemcpyDeviceToHost, c->stream), "diag")) return rc;
    if (int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "diag sync")) return rc;
    const int K = c->last_was_pred ? c->pred_iters
                  : (c->ncg_tol > 0.0 && c->params[0].ncg_iters > 0) ? (int)s[S_NITER] : c->params[0].ncg_iters;
    std::memset(out, 0, sizeof(double) * 24);
    for (int I = 0; I < 3; ++I) {
        out[I] = s[S_MASS0 + I];
        out[3 + I] = s[S_DRIFT0 + I];
    }
    out[6] = s[S_RHO];
    out[7] = s[S_JX]; out[8] = s[S_JY]; out[9] = s[S_JZ];
    out[10] = s[S_UMAX];
    out[11] = s[S_Q];
    out[12] = s[S_QS];
    out[13] = K;
    out[14] = s[S_GG0];
    out[15] = s[S_GMAX0];
    out[16] = K > 0 ? s[S_ITER0 + 4 * (K - 1) + 2] : s[S_GG0];
    out[17] = K > 0 ? s[S_ITER0 + 4 * (K - 1) + 3] : s[S_GMAX0];
    out[18] = (double)c->steps;
    out[19] = (double)c->zc;
    out[20] = (double)c->kfuse;
    out[21] = (double)c->n_pred;
    out[22] = (double)c->n_exact;
    out[23] = c->pred_err;
    return DSCF_OK;
}

int dscf_status(dscf_ctx* c) {
    if (!c) return DSCF_ERR_ARG;
    if (int rc = set_dev(c)) return rc;
    if (int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "status sync")) return rc;
    if (int rc = cuda_check(c, cudaGetLastError(), "status")) return rc;
    int st = 0;
    if (int rc = cuda_check(c, cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost), "status read")) return rc;
    if (st & ST_TIMEOUT) {
        // The sweeps that ran since the timeout skipped their waits (the abort flag was set), so
        // the fields are invalid, but every launch has finished.  Re-arm the brick step counters,
        // the abort flag and the status bit so that the context can be used again once the
        // caller has restored its fields.
        cudaError_t e = cudaMemsetAsync(c->d_status + kFlagBase, 0, sizeof(int) * (size_t)kMaxBricks * kFlagStride, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status + 2, 0, sizeof(int), c->stream);
        const int clear = st & ~(int)ST_TIMEOUT;
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_status, &clear, sizeof(int), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (int rc = cuda_check(c, e, "re-arming after a timeout")) return rc;
        return fail(c, DSCF_ERR_TIMEOUT, "a persistent contour sweep gave up waiting for a neighbour");
    }
    if (st & ST_NONFINITE) return fail(c, DSCF_ERR_NUMERIC, "non-finite value in a reduction");
    return DSCF_OK;
}

int dscf_set_noise(dscf_ctx* c, double omega, int32_t lb_noise, uint64_t seed) {
    if (!c) return DSCF_ERR_ARG;
    if (!(omega >= 0.0) || !std::isfinite(omega)) return fail(c, DSCF_ERR_ARG, "omega must be finite and >= 0");
    if (int rc = set_dev(c)) return rc;
    if (int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "noise sync")) return rc;
    for (int r = 0; r < c->nrep; ++r) {
        Rep& R = c->L.reps[r];
        const dscf_params& q = c->params[r];
        R.noise_amp2 = omega > 0.0 ? 2.0 * q.M * q.dt / omega : 0.0;
        R.noise_kT = (omega > 0.0 && lb_noise) ? q.dt * q.dt / omega : 0.0;
        R.noise_seed = seed;
    }
    if (int rc = cuda_check(c, cudaMemcpyAsync(c->d_reps, c->L.reps.data(), sizeof(Rep) * c->nrep,
                                               cudaMemcpyHostToDevice, c->stream), "noise parameters"))
        return rc;
    if (int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "noise parameters")) return rc;
    c->noise = omega > 0.0 ? (1 | (lb_noise ? 2 : 0)) : 0;
    if (c->exec) {
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
    }
    if (c->exec_pred) {
        cudaGraphExecDestroy(c->exec_pred);
        c->exec_pred = nullptr;
    }
    return DSCF_OK;
}

int dscf_set_warm_start(dscf_ctx* c, int32_t mode) {
    if (!c) return DSCF_ERR_ARG;
    if (mode != 0 && mode != 1) return fail(c, DSCF_ERR_ARG, "mode must be 0 (previous potentials) or 1 (extrapolated)");
    if (int rc = set_dev(c)) return rc;
    if (int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "warm-start sync")) return rc;
    if (c->exec) {
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
    }
    c->warm = mode;
    return reset_warm(c);
}

int dscf_set_inversion_tol(dscf_ctx* c, double tol) {
    if (!c) return DSCF_ERR_ARG;
    if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(c, DSCF_ERR_ARG, "tol must be finite and >= 0");
    if (int rc = set_dev(c)) return rc;
    if (int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "inversion-tolerance sync")) return rc;
    if (c->exec) {
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
    }
    c->ncg_tol = tol;
    return DSCF_OK;
}

int dscf_set_wait_limit(dscf_ctx* c, int32_t polls) {
    if (!c) return DSCF_ERR_ARG;
    if (polls < 1) return fail(c, DSCF_ERR_ARG, "polls must be >= 1");
    if (int rc = set_dev(c)) return rc;
    if (int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "wait-limit sync")) return rc;
    if (c->exec) {
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
    }
    if (c->exec_pred) {
        cudaGraphExecDestroy(c->exec_pred);
        c->exec_pred = nullptr;
    }
    c->wait_limit = polls;
    return DSCF_OK;
}

int dscf_inject_lag(dscf_ctx* c, int32_t brick) {
    if (!c) return DSCF_ERR_ARG;
    if (!c->pers_bz || c->kfuse != 0) return fail(c, DSCF_ERR_STATE, "the context does not run persistent sweeps");
    const int nb = pers_total_bricks(c);
    if (brick < 0 || brick >= nb) return fail(c, DSCF_ERR_ARG, "brick index out of range");
    if (int rc = set_dev(c)) return rc;
    // a counter far behind the others: the brick's neighbours wait for step values it never
    // publishes during the next sweep, the brick itself sees its neighbours ahead and runs through
    const int lag = -(1 << 24);
    cudaError_t e = cudaMemcpyAsync(c->d_status + kFlagBase + (size_t)brick * kFlagStride, &lag, sizeof(int),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_check(c, e, "inject lag");
}

int dscf_probe(dscf_ctx* c, int32_t enable) {
    if (!c) return DSCF_ERR_ARG;
    if (int rc = set_dev(c)) return rc;
    const bool on = enable != 0;
    if (on && !c->ev[0]) {
        for (int i = 0; i < 6; ++i)
            if (int rc = cuda_check(c, cudaEventCreate(&c->ev[i]), "probe event")) return rc;
    }
    if (on != c->probe && c->exec) {
        if (int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "probe sync")) return rc;
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
    }
    c->probe = on;
    c->probe_ran = false;
    return DSCF_OK;
}

int dscf_probe_ms(dscf_ctx* c, float* ms) {
    if (!c || !ms) return DSCF_ERR_ARG;
    if (!c->probe || !c->probe_ran) return fail(c, DSCF_ERR_STATE, "probe not enabled or no step since enabling it");
    if (int rc = set_dev(c)) return rc;
    if (int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "probe sync")) return rc;
    ms[0] = ms[1] = ms[2] = 0.0f;
    if (c->params[0].ncg_iters > 0 && !(c->ncg_tol > 0.0))
        if (int rc = cuda_check(c, cudaEventElapsedTime(&ms[0], c->ev[0], c->ev[1]), "probe sweeps")) return rc;
    if (c->params[0].hydro)
        if (int rc = cuda_check(c, cudaEventElapsedTime(&ms[1], c->ev[2], c->ev[3]), "probe lb")) return rc;
    return cuda_check(c, cudaEventElapsedTime(&ms[2], c->ev[4], c->ev[5]), "probe step");
}

int dscf_set_predictor(dscf_ctx* c, dscf_net* net, int32_t corrector_every, double tol, int32_t ncg_iters) {
    if (!c) return DSCF_ERR_ARG;
    if (int rc = set_dev(c)) return rc;
    if (int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "predictor sync")) return rc;
    if (c->exec_pred) {
        cudaGraphExecDestroy(c->exec_pred);
        c->exec_pred = nullptr;
    }
    if (!net) {
        if (c->last_was_pred) c->phim_stale = true;
        c->net = nullptr;
        return DSCF_OK;
    }
    const Rep& R = c->L.reps[0];
    if (c->prec != DSCF_FP32 || c->nrep != 1 || R.ns != 2)
        return fail(c, DSCF_ERR_ARG, "the learned predictor needs one FP32 melt replica");
    if (!dscf_net_fits(net, R.nx, R.ny, R.nz))
        return fail(c, DSCF_ERR_ARG, "the network context must have this grid and batch 1");
    if (corrector_every < 1 || !(tol > 0.0)) return fail(c, DSCF_ERR_ARG, "need corrector_every >= 1 and tol > 0");
    if (ncg_iters < 0 || ncg_iters > kMaxNcg) return fail(c, DSCF_ERR_ARG, "predictor inversion iterations out of range");
    c->net = net;
    c->pred_iters = ncg_iters > 0 ? ncg_iters : c->params[0].ncg_iters;
    c->pred_k = corrector_every;
    c->pred_tol = tol;
    c->pred_ok = false;
    c->pred_counter = 0;
    c->n_pred = c->n_exact = 0;
    c->pred_err = -1.0;
    return DSCF_OK;
}

int dscf_set_tuning(dscf_ctx* c, int32_t zc, int32_t kfuse) {
    if (!c) return DSCF_ERR_ARG;
    if (zc < 1 || kfuse < 0 || kfuse > 4) return fail(c, DSCF_ERR_ARG, "need zc >= 1 and 0 <= kfuse <= 4");
    if (kfuse > 1 && !c->fusable)
        return fail(c, DSCF_ERR_ARG, "contour fusion needs FP32 and nx in {32, 64, 128} (or 256 for every replica)");
    if (kfuse > 2 && c->L.w8) return fail(c, DSCF_ERR_ARG, "rows of 256 sites fuse at most two contour steps");
    if (kfuse == 0 && !c->pers_bz)
        return fail(c, DSCF_ERR_ARG,
                    "persistent sweeps need FP32 replicas with nx in {32, 48, 64, 96, 128}, ny %% 8 = 0 and nz a "
                    "multiple of the brick depth (16, or 8), and all bricks co-resident");
    int pbz = c->pers_bz, pnw = c->pers_nw;
    if (kfuse == 0 && (zc == 8 || zc == 16)) {   // brick depth requested
        if (zc == 16 && pers_all_supported(c, 16, 16)) { pbz = 16; pnw = 16; }
        else if (zc == 8 && pers_all_supported(c, 8, 8)) { pbz = 8; pnw = 8; }
        else return fail(c, DSCF_ERR_ARG, "no persistent sweep with bricks of %d planes for these grids", zc);
    }
    for (const Rep& R : c->L.reps)
        if (kfuse > R.N) return fail(c, DSCF_ERR_ARG, "kfuse exceeds a chain length");
    if (int rc = set_dev(c)) return rc;
    if (int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "tuning sync")) return rc;
    if (c->exec) {
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
    }
    if (c->exec_pred) {
        cudaGraphExecDestroy(c->exec_pred);
        c->exec_pred = nullptr;
    }
    if (kfuse == 0 && (pbz != c->pers_bz || pnw != c->pers_nw || c->pgroups.empty())) {
        for (const Rep& R : c->L.reps)
            if (int rc = cuda_check(c, (cudaError_t)pers_prepare(R.nx, pers_pby(R), pbz, pnw), "persistent sweep set-up"))
                return rc;
        if (int rc = cuda_check(c, (cudaError_t)pers_prepare(0, 0, pbz, pnw), "persistent sweep set-up")) return rc;
        c->pers_bz = pbz;
        c->pers_nw = pnw;
        if (int rc = reset_pers_flags(c)) return rc;
        if (int rc = place_bricks(c)) return rc;
    }
    c->zc = kfuse == 0 ? c->pers_bz : zc;
    c->kfuse = kfuse;
    set_zc(c, c->zc);
    return upload_tiles(c);
}

int dscf_free(dscf_ctx* c) {
    if (!c) return DSCF_OK;
    cudaSetDevice(c->device);
    for (int i = 0; i < 6; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->exec_pred) cudaGraphExecDestroy(c->exec_pred);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->cap_body) cudaStreamDestroy(c->cap_body);
    delete c;
    return DSCF_OK;
}

const char* dscf_last_error(const dscf_ctx* c) { return c ? c->err.c_str() : g_init_error.c_str(); }

int64_t dscf_launches_per_step(const dscf_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"
