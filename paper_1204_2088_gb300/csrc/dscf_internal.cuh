// Internal declarations of the CUDA library: replica descriptors, partial-sum slots and the
// deterministic block reductions every kernel uses.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dscf {

constexpr int kFlatThreads = 256;     // threads of every site-parallel ("flat") kernel
constexpr int kMaxFlatBlocks = 608;   // flat blocks per replica (= partial sums per replica): 4 per SM, one wave
constexpr int kMaxNcg = 32;           // Fletcher-Reeves iterations per step, upper bound
constexpr int kScalStride = 192;      // FP64 scalar slots per replica
constexpr int kPropCols = 30;         // output x columns per propagator CTA (a warp minus 2 halo lanes)
constexpr int kPropRows = 8;          // output y rows per propagator CTA
// cp.async ring depth of the propagator kernels for an element size
__host__ __device__ constexpr int prop_depth(size_t es) { return es == 8 ? 2 : 4; }

// Partial-sum slots: one array of per-block FP64 partials per slot and replica.  Reducing a
// slot is done redundantly, in a fixed order, by every block that needs the total, so the
// result is bit-identical in all blocks and from run to run.
enum PartSlot {
    P_Q = 0,     // sum_r G_N(r)            (written by the last forward contour step)
    P_ES,        // sum_r exp(-U_S)         (written by the Boltzmann-factor kernel)
    P_H0,        // <g, d>
    P_CD,        // <d, phi_m d>
    P_H1,        // <phi* - phi[U + a1 d], d>
    P_GG0,       // <g, g>, even iterations
    P_GG1,       // <g, g>, odd iterations
    P_GMAX,      // max |g|
    P_MASS0, P_MASS1, P_MASS2,   // sum_r phi_I after the convection-diffusion update
    P_RHO, P_JX, P_JY, P_JZ,     // LB mass and momentum
    P_UMAX,      // max |u_lat|
    P_OBS0, P_OBS1, P_OBS2, P_OBS3, P_OBS4, P_OBS5,   // observables (dscf_observables)
    NPART
};

// Scalar history slots (per replica, FP64).
enum ScalSlot {
    S_GG0 = 0, S_GMAX0 = 1,      // start of the inversion
    S_ITER0 = 2,                 // per iteration k: a1, a, gg, gmax at S_ITER0 + 4k + {0..3}
    S_Q = 160, S_QS, S_DRIFT0, S_DRIFT1, S_DRIFT2, S_MASS0, S_MASS1, S_MASS2,
    S_RHO, S_JX, S_JY, S_JZ, S_UMAX, S_PERR,
    S_NITER,                     // inversion iterations run in the last step (residual stop)
    // totals of partial sums, formed once by the last block of the kernel that wrote them:
    S_H0S, S_CDS, S_H1S,         // line search: <g,d>, <d, phi_m d>, h1
    S_GGS0, S_GGS1,              // <g,g> in the parity slots of the iterations
    S_TOT0, S_TOT1, S_TOT2,      // sum_r phi_I before the mass correction
    S_WARM,                      // steps whose starting potentials Uprev holds (0, 1, 2 = enough)
    S_FIN = kScalStride - 1      // finished-block count (an unsigned in this slot's bytes)
};

// Device status bits.
enum { ST_NONFINITE = 1, ST_TIMEOUT = 2 };
// Layout of the status block: [0] status word, [1] LB step counter, [2] abort flag of the
// persistent sweeps, [3] change flag of the solvent-component labelling, [kFlagBase..] one step
// counter per persistent brick.
constexpr int kFlagBase = 64;
constexpr int kFlagStride = 32;   // ints between brick step counters: one 128-byte line each
constexpr int kMaxBricks = 4096;
// status block: the words above, kMaxBricks counters, then the int4 brick table of the sweeps
constexpr size_t kStatusInts = (size_t)kFlagBase + (size_t)kMaxBricks * kFlagStride + 4 * (size_t)kMaxBricks;

// One replica as the kernels see it.  Pointers are into the caller's workspace; their element
// type is the context precision (double or float) except part/scal (double).
struct Rep {
    int nx, ny, nz, ns, N, nA;
    long long V;
    int tiles_x, tiles_y, tiles_z, zc;     // propagator tiling
    int vec;                               // 1, 2, 4: whole-row layout with nx = 32 vec; 0: tiled
    int tile0, ntiles;
    int blk0, nblk, chunk;                 // flat tiling: nblk blocks of `chunk` sites
    int lb_blk0, lb_nblk;                  // LB grid: one site per thread, lb_nblk blocks
    int hydro, cn_sweeps;
    double phi_p, kappa, alpha, dt, M, gs, gb, rho0, phi_floor;
    double chi[9];
    double mass0[3];
    long long ext_off;                     // offset of this replica in [rep][ns][V] arrays
    long long vbase;                       // sites of the replicas before it ([rep][c][V] arrays)
    void* phi;   // [ns][V] compositions (target of the inversion)
    void* U;     // [ns][V]
    void* mu;    // [ns][V]
    void* d;     // [ns][V] conjugate direction
    void* phim;  // [ns][V] phi[U]
    void* q;     // [2][V]  contour quadratures
    void* E;     // [ns][V] Boltzmann factors exp(-U)
    void* G;     // [N][V]  forward propagators G_1..G_N
    void* Gp0;   // [V]     backward propagator ping
    void* Gp1;   // [V]     backward propagator pong
    void* u;     // [3][V]  LB velocity (lattice units)
    void* pop0;  // [19][V] LB population deviations (post-collision), even steps
    void* pop1;  // [19][V] odd steps
    void* del0;  // [ns][V] Jacobi iterate ping
    void* del1;  // [ns][V] Jacobi iterate pong
    void* rhs;   // [ns][V] right-hand side of the Crank-Nicolson system
    void* Uprev; // [ns][V] potentials the previous step's inversion started from
    // thermal noise (dscf_set_noise): composition flux variance 2 M dt / Omega per unit phi,
    // LB temperature dt^2 / Omega (0: off), generator key
    double noise_amp2, noise_kT;
    unsigned long long noise_seed;
    int rep_index;                         // counter word 3 of the noise (replica in the batch)
    double* part;   // [NPART][part_stride]
    int part_stride;
    double* scal;   // [kScalStride]
};

// Propagator and flat tiling of one replica for a given z-chunk; the context path and the
// allocation-free path both use it.
// rows256: every replica of the launch has rows of 256 sites, which then take the whole-row
// contour kernels of their own (8 sites per lane); otherwise such rows take the tiled layout.
inline void tile_replica(Rep& R, int zc, bool rows256 = false) {
    R.vec = (R.nx == 32 || R.nx == 64 || R.nx == 128) ? R.nx / 32 : ((rows256 && R.nx == 256) ? 8 : 0);
    R.tiles_x = R.vec ? 1 : (R.nx + kPropCols - 1) / kPropCols;
    R.tiles_y = (R.ny + kPropRows - 1) / kPropRows;
    R.zc = zc < 1 ? 1 : (zc > R.nz ? R.nz : zc);
    R.tiles_z = (R.nz + R.zc - 1) / R.zc;
    R.ntiles = R.tiles_x * R.tiles_y * R.tiles_z;
    long long nb = (R.V + kFlatThreads - 1) / kFlatThreads;
    if (nb > kMaxFlatBlocks) nb = kMaxFlatBlocks;
    long long chunk = (R.V + nb - 1) / nb;
    chunk = (chunk + kFlatThreads - 1) / kFlatThreads * kFlatThreads;
    R.chunk = (int)chunk;
    R.nblk = (int)((R.V + chunk - 1) / chunk);
    R.lb_nblk = (int)((R.V + kFlatThreads - 1) / kFlatThreads);
}
constexpr int kMinZc = 4;             // smallest z-chunk the autotuner tries (most tiles)

// Launch description shared by the host launchers.
struct Launch {
    const Rep* reps;         // device table
    const int* tile2rep;     // device map: propagator tile -> replica
    const int* blk2rep;      // device map: flat block -> replica
    int* status;             // device status word
    int* counter;            // device step counter (selects the LB buffer parity)
    int nblk_total;          // flat blocks over all replicas
    int nlb_total;           // LB blocks over all replicas
    int nrep;
    int noise;               // thermal noise: 1 compositions, 2 LB modes
    cudaStream_t stream;
    int w8 = 0;              // every replica in whole rows of 256 sites (their own contour kernels)
};

// ---------------------------------------------------------------------------------------------
// Deterministic reductions (warp shuffle then one warp over the warp sums).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum; the result is returned to every thread.  sh: >= 33 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int l = tid & 31, w = tid >> 5;
    (void)lane; (void)warp;
    v = warp_sum(v);
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        double x = (l < nw) ? sh[l] : 0.0;
        x = warp_sum(x);
        if (l == 0) sh[32] = x;
    }
    __syncthreads();
    double r = sh[32];
    __syncthreads();
    return r;
}

// NV block-wide sums in one pass (same order per value as block_sum, so the same results).
// sh: >= 33 NV doubles of shared memory.
template <int NV>
__device__ __forceinline__ void block_sum_n(double (&v)[NV], double* sh) {
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int l = tid & 31, w = tid >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        v[k] = warp_sum(v[k]);
        if (l == 0) sh[33 * k + w] = v[k];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = (l < nw) ? sh[33 * k + l] : 0.0;
            x = warp_sum(x);
            if (l == 0) sh[33 * k + 32] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = sh[33 * k + 32];
    __syncthreads();
}

__device__ __forceinline__ double block_max(double v, double* sh) {
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int l = tid & 31, w = tid >> 5;
    v = warp_max(v);
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        double x = (l < nw) ? sh[l] : 0.0;
        x = warp_max(x);
        if (l == 0) sh[32] = x;
    }
    __syncthreads();
    double r = sh[32];
    __syncthreads();
    return r;
}

// Total of n partials, same fixed order in every block.
__device__ __forceinline__ double reduce_parts(const double* __restrict__ p, int n, double* sh) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nt = blockDim.x * blockDim.y;
    double s = 0.0;
    for (int i = tid; i < n; i += nt) s += p[i];
    return block_sum(s, sh);
}
// Totals of NV partial arrays of n entries each, in one pass (same results as reduce_parts).
template <int NV>
struct Parts {
    const double* p[NV];
};
template <int NV>
__device__ __forceinline__ void reduce_parts_n(const Parts<NV> p, int n, double (&out)[NV], double* sh) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nt = blockDim.x * blockDim.y;
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = 0.0;
    for (int i = tid; i < n; i += nt)
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] += p.p[k][i];
    block_sum_n<NV>(out, sh);
}
// The same totals read through L2 (ld.global.cg), for partials that other blocks of the running
// kernel have just written.
__device__ __forceinline__ double reduce_parts_cg(const double* p, int n, double* sh) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nt = blockDim.x * blockDim.y;
    double s = 0.0;
    for (int i = tid; i < n; i += nt) s += __ldcg(p + i);
    return block_sum(s, sh);
}
template <int NV>
__device__ __forceinline__ void reduce_parts_n_cg(const Parts<NV> p, int n, double (&out)[NV], double* sh) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nt = blockDim.x * blockDim.y;
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = 0.0;
    for (int i = tid; i < n; i += nt)
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] += __ldcg(p.p[k] + i);
    block_sum_n<NV>(out, sh);
}
__device__ __forceinline__ double reduce_parts_max(const double* __restrict__ p, int n, double* sh) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nt = blockDim.x * blockDim.y;
    double s = 0.0;
    for (int i = tid; i < n; i += nt) s = fmax(s, p[i]);
    return block_max(s, sh);
}

__device__ __forceinline__ double* slot(const Rep& R, int s) { return R.part + (size_t)s * R.part_stride; }

// Fence-and-count: after thread 0 of every block of the replica has written its partials, true in
// the one block that finishes last, where every block's partials are visible.  The count wraps
// to zero at R.nblk, so it is ready for the next launch without a reset.  The last block forms
// the totals once (in the same order as reduce_parts), instead of every block of the consuming
// kernel re-reading all partials of one L2 line set.
__device__ __forceinline__ bool last_block_of(const Rep& R, int* flag_sh) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned old = atomicInc((unsigned*)(R.scal + S_FIN), (unsigned)R.nblk - 1u);
        *flag_sh = (old == (unsigned)R.nblk - 1u);
    }
    __syncthreads();
    const bool last = *flag_sh != 0;
    if (last) __threadfence();
    return last;
}

__device__ __forceinline__ int wrapi(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// Boltzmann factor exp(-x) in the field precision (CUDA's exp / expf, not re-implemented).
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each multiplies counter words 0
// and 2 by 0xD2511F53 and 0xCD9E8D57 (32 x 32 -> 64 bits), XORs the high halves into words 1 and
// 3 with the key, and swaps; the key advances by the Weyl constants 0x9E3779B9, 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, unsigned k0, unsigned k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}
// Four standard normals of counter (site, step, stream, replica): uniforms (top 24 bits + 1/2) /
// 2^24, Box-Muller on words (0, 1) and (2, 3).
template <typename T>
__device__ __forceinline__ void normals4(unsigned long long seed, unsigned site, unsigned step, unsigned stream,
                                         unsigned rep, T (&n)[4]) {
    const uint4 r = philox4x32_10(make_uint4(site, step, stream, rep), (unsigned)seed, (unsigned)(seed >> 32));
    const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
        const T ua = ((T)(w[2 * pr] >> 8) + T(0.5)) * T(1.0 / 16777216.0);
        const T ub = ((T)(w[2 * pr + 1] >> 8) + T(0.5)) * T(1.0 / 16777216.0);
        T sn, cs;
        if constexpr (sizeof(T) == 4) {
            const float rad = sqrtf(-2.f * logf(ua));
            sincospif(2.f * ub, &sn, &cs);
            n[2 * pr] = rad * cs;
            n[2 * pr + 1] = rad * sn;
        } else {
            const double rad = sqrt(-2.0 * log(ua));
            sincospi(2.0 * ub, &sn, &cs);
            n[2 * pr] = rad * cs;
            n[2 * pr + 1] = rad * sn;
        }
    }
}

__device__ __forceinline__ double bexp(double x) { return exp(-x); }
__device__ __forceinline__ float bexp(float x) { return expf(-x); }

// ---------------------------------------------------------------------------------------------
// Host launchers (defined in the kernel translation units, explicit per precision).
// ---------------------------------------------------------------------------------------------
template <typename T> void launch_prop_fwd(const Launch& L, int s, int grid, size_t smem);
template <typename T> void launch_prop_bwd(const Launch& L, int j, int grid, size_t smem);
template <typename T> int prop_set_smem_limit(size_t bytes);   // returns a cudaError_t
size_t prop_smem_bytes(int vec, bool bwd, size_t es);           // dynamic shared memory of one CTA
// fused contour groups of K steps (FP32, whole-row layout only)
size_t prop_fused_smem_bytes(int vec, int K);
void launch_prop_fused(const Launch& L, bool bwd, int K, int g, int grid, size_t smem);
int prop_fused_set_smem_limit(size_t bytes);                    // returns a cudaError_t
// mode: 0 exp(-U), 1 trial exp(-(U + a1 d)), 2 commit U += a d then exp(-U), 3 exp(-Uext)
template <typename T> void launch_exp(const Launch& L, int mode, int k, const void* Uext, int write_u = 0);
// net != 0: the density at the evaluated potential is the learned predictor's output, stored in q
template <typename T> void launch_trial(const Launch& L, int net = 0);
template <typename T> void launch_grad(const Launch& L, int k, int net = 0);
// Residual stop of the inversion before iteration k: sets the graph condition `handle` to 1 while
// max|g| >= tol for some replica (0 otherwise, also for a non-finite residual) and records the
// iterations run in scal[S_NITER]; k = 0 also records the start-of-inversion residual.
void launch_ncg_gate(const Launch& L, int k, double tol, unsigned long long handle);
void launch_pred_err(const Launch& L);   // max |q - phi_m| of replica 0 into scal[S_PERR] (FP32 melts)
// Observables: pass 1 leaves per-block sums of phi_I (slots P_OBS0..2), U.phi (P_OBS3) and the
// interaction energy density (P_OBS4); pass 2, given the species means, sum (phi_I - <phi_I>)^2
// over I (P_OBS0) and |phi_A + phi_B - <phi_A> - <phi_B>| (P_OBS1).
template <typename T>
void launch_obs1(const Launch& L);
template <typename T>
void launch_obs2(const Launch& L, double mA, double mB, double mS);
// per-block counts of cubes, faces, edges, vertices of {phi_species > threshold} into P_OBS0..3
template <typename T> void launch_minkowski(const Launch& L, int replica, int species, double threshold);
// trapped solvent: component labels of the complement of {phi_B > threshold} (lab, cnt: V ints)
template <typename T> void launch_cc_init(const Launch& L, int replica, double threshold, int* lab, int* cnt);
void launch_cc_step(const Launch& L, int replica, int* lab, int* changed);
void launch_cc_count(const Launch& L, int replica, const int* lab, int* cnt);   // P_OBS0/1 largest size/root, P_OBS4 roots
template <typename T> void launch_cc_solvent(const Launch& L, int replica, const int* lab, int bulk);   // P_OBS2, 3
// mode 0: init (d = -g), mode 1: iteration k direction update
template <typename T> void launch_dir(const Launch& L, int mode, int k);
template <typename T> void launch_mu(const Launch& L, int K);   // K < 0: iterations from scal[S_NITER]
template <typename T> void launch_extrap(const Launch& L);       // extrapolated start of the inversion
template <typename T> void launch_lb(const Launch& L, const void* force_ext);
template <typename T> void launch_cd(const Launch& L, int sweeps);
template <typename T> void launch_dens_out(const Launch& L, void* phi_ext);
template <typename T> void launch_pop_copy(const Launch& L, void* ext, int dir);  // 0 get, 1 set
template <typename T> void launch_mass_init(const Launch& L, int nrep);
void launch_step_end(const Launch& L);
template <typename T> void launch_lb_diag(const Launch& L);
// persistent contour sweeps (FP32; row widths 32, 48, 64, 96, 128; several replicas of one width
// per launch, each CTA taking its brick from an int4 table: replica, brick in the replica, flag
// index of the replica's brick 0)
// Brick rows: 16 for rows of at most 64 sites (so that a brick, and the co-resident launch, holds
// as many sites as for the wider rows) where ny allows it, else 8.
__host__ __device__ inline int pers_pby_of(int nx, int ny) { return (nx <= 64 && ny % 16 == 0) ? 16 : 8; }
size_t pers_smem_bytes(int width, int pby, int bz);
size_t pers_mix_smem_bytes(int bz);                            // the mixed-width launches (width 0)
bool pers_width_ok(int nx);
int pers_pby(const Rep& R);                                    // brick rows of a replica (8 or 16)
bool pers_supported(const Rep& R, int bz, int nw, int nsm);   // nw: warps per CTA (16, or 8 with 2 CTAs per SM)
int pers_bricks(const Rep& R, int bz);
int pers_prepare(int width, int pby, int bz, int nw);   // cudaError_t; width 0: the mixed-width kernel
// width 0: bricks of several widths in one launch (bricks of 16 planes)
int launch_prop_pers(const Launch& L, bool bwd, int width, int pby, int bz, int nw, int nbricks, const int4* table,
                     int* flags, int* abortf, int limit);  // cudaError_t
// SM id of each CTA of a sweep-shaped cooperative launch (cudaError_t)
int pers_placement(int bz, int nw, int nbricks, int* d_smid, cudaStream_t stream);

}  // namespace dscf

namespace dscf {
// tcgen05 forward convolution of the predictor network (dscf_tc.cu)
bool tc_conv_supported(int nx, int ny);
size_t tc_conv_smem();
int tc_conv_prepare();   // cudaError_t
int tc_conv_blocks(int nx, int ny, int nz);   // CTAs per sample
void launch_conv_tc(int layer, const void* in, const void* wt, const float* bias, int cout, void* out, int nx, int ny,
                    int nz, int B, double* part, int* err, cudaStream_t s);
}  // namespace dscf
// learned predictor (dscf_net.cu): forward pass on a given stream, for use inside the step graph
struct dscf_net;
bool dscf_net_fits(const dscf_net* net, int nx, int ny, int nz);
int dscf_net_forward_launches(const dscf_net* n);   // kernels one forward pass launches
void dscf_net_forward_on(dscf_net* net, cudaStream_t stream, const float* U, double pb0, double pb1, float* phi);
