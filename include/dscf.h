/*
 * dscf.h -- C ABI of the GB300 (sm_103a) hot path of the hybrid lattice-Boltzmann / dynamic
 * self-consistent-field method (Zhang, Sevink, Schmid, arXiv:1204.2088).
 *
 * One time step (Sec. 2, paragraph after Eq. 17: "LB steps alternate with propagations of
 * Eq. (3)", each propagation needing the self-consistent potentials) is:
 *   1. potentials U^n from the compositions phi^n by Fletcher-Reeves nonlinear CG on the
 *      convex functional L(U) = (phi_p V/N) ln Q[U] + phi_s V ln<exp(-U_S)> + sum U phi^n,
 *      whose gradient is phi^n - phi[U]; every gradient needs the Green propagators of
 *      Eq. 17 (27-point linkage stencil) and the contour quadrature of Eq. 16;
 *   2. chemical potentials mu^n, Eq. 4;
 *   3. (hydro) one D3Q19 MRT lattice-Boltzmann collide-stream, Eq. 9-14 / Table 1, driven by
 *      the body force f = -sum_I phi_I grad mu_I of Eq. 8;
 *   4. convection-diffusion update of the compositions, Eq. 3: two-step Lax-Wendroff
 *      convection by the LB velocity, Crank-Nicolson diffusion (Jacobi sweeps), FP64 mass
 *      correction.
 *
 * Conventions.
 *   - Lattice spacing h = 1, energies in k_B T, time in tau = h^2/(k_B T M) (Sec. 2 units).
 *   - Fields are contiguous arrays, x fastest: index x + nx*(y + ny*z); several species are
 *     stored species-major [I][V] in the order A, B, S.  Several replicas are stored one after
 *     the other, replica-major, each with its own V = nx*ny*nz.
 *   - The floating-point type of every field pointer is the context precision: double for
 *     DSCF_FP64, float for DSCF_FP32.  Scalars, the partition function Q, all mass / momentum
 *     sums and the line-search dot products are FP64 in both precisions.
 *   - LB populations are exchanged as deviations n_i - w_i rho0 from the rest equilibrium, in
 *     D3Q19 order 0:(000), 1..6: +x -x +y -y +z -z, 7..18: (+x+y) (-x-y) (+x-y) (-x+y) (+x+z)
 *     (-x-z) (+x-z) (-x+z) (+y+z) (-y-z) (+y-z) (-y+z), as the populations n_i(r, t) that enter
 *     the next collision (Eq. 10 left-hand side).
 *   - LB runs in lattice units (Delta t_LB = 1, c_s^2 = 1/3); the force enters as dt^2 f and
 *     the velocity u_lat = dt u is the Courant number the convection step uses.
 *
 * Memory and streams.  The library allocates no device memory: the caller passes one device
 * workspace of at least dscf_workspace_bytes() bytes (256-byte aligned), which must outlive
 * the context, and a CUDA stream (NULL = legacy default stream).  Every call is asynchronous
 * on that stream unless stated otherwise.  The library owns only host-side bookkeeping plus
 * one CUDA graph and one capture stream, released by dscf_free.
 *
 * Errors.  Every entry point returns DSCF_OK (0) or a negative code; it never aborts and
 * never traps.  dscf_last_error() gives a message.  Device-side problems (non-finite sums) set
 * a device status word that dscf_status() reads.
 */
#ifndef DSCF_H
#define DSCF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    DSCF_OK = 0,
    DSCF_ERR_ARG = -1,      /* invalid argument or parameter                           */
    DSCF_ERR_CUDA = -2,     /* a CUDA runtime call failed                             */
    DSCF_ERR_OOM = -3,      /* the workspace passed is too small                       */
    DSCF_ERR_TIMEOUT = -4,  /* a bounded device wait gave up                           */
    DSCF_ERR_NUMERIC = -5,  /* non-finite value in a reduction (status word)           */
    DSCF_ERR_STATE = -6,    /* call not valid in the current context state             */
    DSCF_ERR_NOCONVERGE = -7 /* a bounded host-driven iteration did not settle          */
};

enum { DSCF_FP64 = 0, DSCF_FP32 = 1 };

/* Field selectors for dscf_get_fields / dscf_set_fields. */
enum {
    DSCF_FIELD_PHI = 0,   /* compositions phi_I            [ns][V]                      */
    DSCF_FIELD_U = 1,     /* potentials U_I                [ns][V]                      */
    DSCF_FIELD_MU = 2,    /* chemical potentials mu_I      [ns][V]  (get only)          */
    DSCF_FIELD_VEL = 3,   /* LB velocity u_lat (Eq. 9)     [3][V]   (get only)          */
    DSCF_FIELD_POP = 4,   /* LB population deviations      [19][V]                      */
    DSCF_FIELD_PHIM = 5   /* phi[U] of the current U       [ns][V]  (get only)          */
};

/*
 * Parameters of one replica (Sec. 2 model and units; Sec. 3 workloads).
 *   nx, ny, nz   periodic lattice (h = 1), each >= 1
 *   ns           2 = A,B melt; 3 = A,B copolymer plus single-bead solvent S (Eq. 2, 3rd line)
 *   N, nA        beads per chain N_p and A-block length n, 1 <= nA < N (bead s is A iff s <= nA)
 *   phi_p        mean copolymer volume fraction (1 in a melt); the solvent takes 1 - phi_p
 *   chi[9]       Flory-Huggins chi_IJ (row-major 3x3, symmetric, zero diagonal), Sec. 2
 *   kappa        Helfand compressibility kappa_H v0 / k_B T (paper: 10)
 *   a            statistical segment length in h (paper: 1.1543); the 27-point linkage
 *                stencil is the tensor product of (alpha, 1 - 2 alpha, alpha), alpha = a^2/6,
 *                which has the per-axis variance a^2/3 of a Gaussian bond; needs alpha < 1/2
 *   dt, M        time step in tau and mobility (paper: M = 1)
 *   tau_s, tau_b LB shear / bulk relaxation times; gamma = 1 - 1/tau (Eq. 13, 15); > 1/2
 *   rho0         LB reference mass density (1)
 *   hydro        0: diffusion only (u = 0); 1: LB coupled
 *   ncg_iters    Fletcher-Reeves iterations per step (fixed count, 0..32)
 *   cn_sweeps    Jacobi sweeps of the Crank-Nicolson system (even, 2..64)
 *   phi_floor    floor on phi inside the local curvature of mu (e.g. 1e-6)
 */
typedef struct {
    int32_t nx, ny, nz;
    int32_t ns;
    int32_t N, nA;
    double phi_p;
    double chi[9];
    double kappa;
    double a;
    double dt, M;
    double tau_s, tau_b, rho0;
    int32_t hydro;
    int32_t ncg_iters;
    int32_t cn_sweeps;
    double phi_floor;
} dscf_params;

typedef struct dscf_ctx dscf_ctx;

/* Bytes of device workspace needed for n_replicas replicas with parameters p[0..n-1] in the
 * given precision.  Returns 0 if the parameters are invalid. */
size_t dscf_workspace_bytes(const dscf_params* p, int32_t n_replicas, int32_t precision);

/*
 * Create a context.  p: n_replicas parameter sets (host memory, copied).  workspace: device
 * pointer (caller-owned, 256-byte aligned, >= dscf_workspace_bytes).  stream: cudaStream_t or
 * NULL.  The initial state is phi = homogeneous melt/solution, U = 0, LB at rest; set the
 * compositions with dscf_set_fields before stepping.  Synchronises the stream once.
 * Errors: DSCF_ERR_ARG (bad parameters), DSCF_ERR_OOM (workspace too small), DSCF_ERR_CUDA.
 */
int dscf_init(const dscf_params* p, int32_t n_replicas, int32_t precision, void* workspace,
              size_t workspace_bytes, void* stream, dscf_ctx** out);

/* dscf_init with a given tuning instead of the autotuner (zc, kfuse as in dscf_set_tuning, for
 * instance the values dscf_diagnostics reported after an earlier dscf_init on the same replica
 * shapes and device): no timing runs.  zc < 0 runs the autotuner (= dscf_init).  DSCF_ERR_ARG if
 * the tuning is not valid for these replicas. */
int dscf_init_tuned(const dscf_params* p, int32_t n_replicas, int32_t precision, void* workspace,
                    size_t workspace_bytes, void* stream, int32_t zc, int32_t kfuse, dscf_ctx** out);

/* Advance every replica by n_steps coupled time steps (steps 1-4 above).  The step sequence
 * is captured once into a CUDA graph and launched n_steps times on the context stream. */
int dscf_step(dscf_ctx* ctx, int32_t n_steps);

/* Forward density map alone (Eq. 2 via Eq. 16-17): phi_out = phi[U_in], for every replica.
 * U_in, phi_out: device pointers, [rep][ns][V] in the context precision.  Does not touch the
 * context's U or phi (uses its propagator buffers). */
int dscf_densities(dscf_ctx* ctx, const void* U_in, void* phi_out);

/* n_steps LB collide-stream steps alone (Eq. 9-14).  force: device pointer [rep][3][V] of
 * lattice-unit body force, or NULL for the thermodynamic force of the current phi and mu. */
int lb_step(dscf_ctx* ctx, const void* force, int32_t n_steps);

/* Copy a field out of / into the context.  on_host != 0: dst/src is host memory (the call
 * synchronises the stream before returning for gets); otherwise device memory.  Setting PHI
 * also sets the per-species mass targets of the mass correction to the new totals; setting U
 * makes the next step recompute phi[U]. */
int dscf_get_fields(dscf_ctx* ctx, int32_t which, void* dst, int32_t on_host);
int dscf_set_fields(dscf_ctx* ctx, int32_t which, const void* src, int32_t on_host);

/* FP64 diagnostics of one replica (synchronises).  out[0..23]:
 *  0..2  sum_r phi_I after the last step, 3..5 its drift before the mass correction,
 *  6 LB mass sum_r rho, 7..9 LB momentum after the last collision, 10 max |u_lat|
 *  (6..10 are reduced from the current populations and velocity when this is called),
 *  11 Q of the last gradient evaluation, 12 <exp(-U_S)>, 13 NCG iterations per step,
 *  14 <g,g> and 15 max|g| at the start of the last inversion, 16 <g,g> and 17 max|g|
 *  at its end, 18 steps done, 19 z-chunk of the propagator tiles (the brick depth when 20 is 0)
 *  and 20 contour steps fused per propagator launch (0: persistent sweeps), as chosen at
 *  dscf_init or by dscf_set_tuning, 21 steps taken with the
 *  learned predictor and 22 exact steps since dscf_set_predictor, 23 the predictor's last
 *  judged error (see dscf_set_predictor; -1 before the first judgement).  Slots 13, 16 and 17
 *  follow the inversion of the last step taken (a predictor step may use fewer iterations). */
int dscf_diagnostics(dscf_ctx* ctx, int32_t replica, double* out);

/* Observables of replica `replica` at the current state (Sec. 3; Eq. 1 restated in volume
 * fractions with constants dropped): out[0] free energy per site
 *   F = -(phi_p / N) ln Q - (1 - phi_p) ln <e^{-U_S}> - <sum_I U_I phi_I>
 *       + <1/2 sum_IJ chi_IJ phi_I sigma[phi_J] + kappa/2 (sum_I phi_I - 1)^2>
 * with Q from an exact density evaluation at the current U (the solvent term only with three
 * species); out[1] order parameter S = sqrt(<sum_I (phi_I - <phi_I>)^2>) (Fig. 1); out[2]
 * segregation <|phi_A + phi_B - <phi_A> - <phi_B>|> (Fig. 3).  Sums in FP64 from per-block
 * partials in a fixed order.  Runs one density evaluation and synchronises the stream. */
int dscf_observables(dscf_ctx* ctx, int32_t replica, double* out);

/* Minkowski functionals of the morphology (Sec. 3, the algorithm of Michielsen and De Raedt): the
 * body is the union of the closed unit cubes of the sites where phi_species > threshold (compared
 * in the context precision; periodic box).  counts[0..3] (host memory) receive its numbers of
 * distinct cubes n_c, faces n_f, edges n_e and vertices n_v, from which V = n_c,
 * S = -6 n_c + 2 n_f, 2B = 3 n_c - 2 n_f + n_e and chi = -n_c + n_f - n_e + n_v (the Euler
 * number of the bounding surfaces, the paper's convention, is 2 chi).  Integer counts, exact.
 * Synchronises.  DSCF_ERR_ARG for a bad replica, species or threshold. */
int dscf_minkowski(dscf_ctx* ctx, int32_t replica, int32_t species, double threshold, int64_t* counts);

/* Trapped solvent (Sec. 3, solvent enclosed by the vesicles as a fraction of all solvent): the
 * aggregates are the body {phi_B > threshold}; its complement splits into face-connected
 * components of the periodic box (found on the device by label propagation to a fixed point);
 * the largest is the bulk outside (ties: the one containing the smallest site index), the others
 * are enclosed.  out[0] = sum of phi_S over the enclosed components / sum of phi_S, out[1] = the
 * number of components.  Solutions only (three species).  Uses the contour stack (recomputed by
 * every density evaluation) as scratch.
 * Synchronises.  DSCF_ERR_ARG without solvent, DSCF_ERR_NOCONVERGE if the labelling does not
 * settle within 64 (nx + ny + nz) + 1024 sweeps. */
int dscf_trapped_solvent(dscf_ctx* ctx, int32_t replica, double threshold, double* out);

/* Synchronise the stream and return the device status word as an error code (DSCF_OK,
 * DSCF_ERR_TIMEOUT if a persistent sweep gave up a bounded wait, DSCF_ERR_NUMERIC) or
 * DSCF_ERR_CUDA if a kernel failed. */
int dscf_status(dscf_ctx* ctx);

/* Release host-side state (graph, capture stream).  The workspace stays the caller's. */
int dscf_free(dscf_ctx* ctx);

/* Message of the last error on this context (or of the last failed dscf_init if ctx NULL). */
const char* dscf_last_error(const dscf_ctx* ctx);

/* Number of kernels one dscf_step(ctx, 1) launches (for launch accounting). */
int64_t dscf_launches_per_step(const dscf_ctx* ctx);

/* Override the autotuner's choice (for instance with a value cached from an earlier run):
 * zc = z planes per propagator tile (>= 1), kfuse = contour steps per propagator launch (1..4;
 * > 1 needs FP32 and nx in {32, 64, 128} for every replica, or nx = 256 for every replica with
 * kfuse <= 2 (rows of 256 sites have contour kernels of their own), and kfuse <= N), or kfuse = 0 for
 * persistent sweeps (FP32; every replica with nx in {32, 48, 64, 96, 128} and ny a multiple of 8;
 * bricks of nx x 8 x 16 sites (nx x 16 x 16 for rows of at most 64 sites where ny allows), one
 * CTA of 16 warps per SM, or of nx x 8 x 8 (nx x 16 x 8) sites, two CTAs of 8 warps per SM; nz a
 * multiple of the brick depth; one warp per plane; replicas share cooperative launches while
 * their bricks fit the SMs together, so a batch takes a few launches per sweep direction).  With
 * kfuse = 0, zc = 16 or 8 selects the brick depth (DSCF_ERR_ARG if the grids do not allow it),
 * any other zc keeps the current depth.  Synchronises the stream; the
 * next dscf_step re-captures its graph.  Results do not depend on either value beyond rounding. */
int dscf_set_tuning(dscf_ctx* ctx, int32_t zc, int32_t kfuse);

/* Thermal noise (Sec. 2: the stochastic term of Eq. 3 with the covariance of Eq. 5, and phi_k r_k in
 * the relaxation of the LB modes, Eq. 13).  omega = 0 (the default) turns it off; omega > 0 is
 * the noise parameter Omega = h^3 / v0 (paper: 400, or 100).  Compositions: minus the divergence of
 * a random flux on every lattice face, variance 2 M phi_face / (Omega dt), added to the explicit
 * part of the Crank-Nicolson step (every species' total is kept).  lb_noise != 0 also draws the
 * fluctuating collision: every non-conserved mode k = 4..18 gains sqrt(rho kT b_k (1 - gamma_k^2)
 * / c_s^2) r_k with the lattice temperature kT = dt^2 / Omega.  Normals: Philox4x32-10 keyed by
 * seed (low word, high word), counter (site, step, stream, replica) with stream 1 + I for species
 * I and 16..19 for the LB modes, uniforms (top 24 bits + 1/2) / 2^24, Box-Muller; the step index
 * is the context's step counter (it starts at 0 and advances once per coupled step and per
 * lb_step).  Synchronises and re-captures the step graph.  DSCF_ERR_ARG for a negative or
 * non-finite omega. */
int dscf_set_noise(dscf_ctx* ctx, double omega, int32_t lb_noise, uint64_t seed);

/* Residual stop of the inversion (step 1): with tol > 0 the Fletcher-Reeves iterations of each
 * exact step stop before iteration k once max_r |phi*_I(r) - phi_I[U](r)| < tol for every replica
 * (or the residual is not finite, which also sets the non-finite status bit), and after at most
 * ncg_iters iterations in any case; tol = 0 (the default) runs exactly ncg_iters iterations.  The
 * decision is taken on the device: every iteration is an IF node of the step's CUDA graph whose
 * condition a one-block kernel sets from the residual the previous iteration left, so a step still
 * costs one graph launch and no host synchronisation.  Diagnostics slot 13 then reports the
 * iterations run in the last step; dscf_launches_per_step counts every possible launch, and the
 * probe's sweep time (dscf_probe_ms, ms[0]) is not measured.  Steps of the learned predictor
 * keep their fixed count.  Synchronises and re-captures the step graph.  DSCF_ERR_ARG for a
 * negative or non-finite tol, DSCF_ERR_CUDA if the graph cannot be built. */
int dscf_set_inversion_tol(dscf_ctx* ctx, double tol);

/* Starting point of the inversion (step 1; the paper does not give it).  mode 0 (the default): the
 * previous step's potentials U^{n-1}.  mode 1: their linear extrapolation in time,
 * 2 U^{n-1} - U^{n-2}, once two steps since the last dscf_set_fields of PHI or U have produced
 * potentials (before that, U^{n-1}); the densities at the starting point are evaluated first, one
 * extra density evaluation per step.  The extrapolation makes the starting residual second order in
 * dt instead of first, so with the residual stop (dscf_set_inversion_tol) fewer iterations are
 * needed; the potentials the inversion converges to do not depend on the start.  Synchronises and
 * re-captures the step graph.  DSCF_ERR_ARG for another mode. */
int dscf_set_warm_start(dscf_ctx* ctx, int32_t mode);

/* Failure detection of the persistent sweeps.  Every wait of a persistent sweep on a
 * neighbouring brick is bounded by `polls` polls (default 4194304, several seconds; each poll is
 * an acquire load of the neighbour's step counter followed by a short sleep).  A CTA that runs out
 * sets the status bit and a global abort flag; every other CTA then stops waiting, all launches
 * finish, and dscf_status reports DSCF_ERR_TIMEOUT.  That call also re-arms the step counters, so
 * the context stays usable once the caller has restored its fields (they are invalid after a
 * timeout).  dscf_set_wait_limit synchronises and re-captures the step graph.
 * dscf_inject_lag (test hook, host side: one 4-byte copy) sets brick `brick`'s step counter far
 * behind the others, so that during the next persistent sweep its neighbours wait for values it
 * never publishes and run out of polls.  Bricks are numbered replica by replica (in the order
 * of the replicas), y fastest, then z.  DSCF_ERR_STATE unless the context uses persistent sweeps
 * (kfuse 0), DSCF_ERR_ARG for a brick outside 0 .. bricks-1 (all replicas) or polls < 1. */
int dscf_set_wait_limit(dscf_ctx* ctx, int32_t polls);
int dscf_inject_lag(dscf_ctx* ctx, int32_t brick);

/* Measured fused multiply-add throughput of the CUDA cores of the current device, in the given
 * precision (a measurement helper for the arithmetic roofline of the kernels above; the paper has
 * no counterpart): eight independent FMA chains per thread on 8 CTAs of 256 threads per SM, timed
 * with CUDA events on `stream` (cudaStream_t or NULL), the best of three runs after a warm-up run
 * (each a few tens of milliseconds).  *tflops receives 2 x FMAs / second / 1e12.  Synchronises the
 * stream.  DSCF_ERR_ARG for a bad precision or NULL output, DSCF_ERR_CUDA if a launch fails. */
int dscf_fma_peak(int32_t precision, void* stream, double* tflops);

/* Timing probe.  enable != 0 makes the next dscf_step capture CUDA events (created by the
 * library) into the step graph: around the 2N contour-sweep launches of the first gradient
 * evaluation of the step, around the LB collide-stream launch, and around the whole step.
 * dscf_probe_ms synchronises the stream and returns, for the most recent step, the elapsed
 * milliseconds of those three regions (ms[0] sweeps, ms[1] LB, ms[2] step); regions that did
 * not run read 0.  DSCF_ERR_STATE if the probe is off or no step ran since enabling it. */
int dscf_probe(dscf_ctx* ctx, int32_t enable);
int dscf_probe_ms(dscf_ctx* ctx, float* ms);

/*
 * Forward density map phi_out = phi[U_in] for one replica, for callers that cannot allocate
 * device memory at all (a host framework that owns every device allocation, a callback in
 * which allocation is forbidden, a process whose device footprint is fixed after start-up) and
 * therefore cannot supply the workspace dscf_init needs.  The paper has no counterpart: this
 * is an interface for such callers, computing the same map as dscf_densities.
 *
 * p: parameters of one replica (host memory; only the chain, stencil and composition fields
 * matter).  U_in, phi_out: device pointers, [ns][V] in the given precision; their device is the
 * one used (the call switches to it and restores the calling thread's current device before it
 * returns).  stream: cudaStream_t or NULL, a stream of that device.  Asynchronous on the stream.
 *
 * Neither the library nor the caller allocates anything: all scratch (propagator stack,
 * Boltzmann factors, quadratures, partial sums) lives in one file-scope device array of
 * DSCF_STATIC_SCRATCH_BYTES, which every GPU that loads the library holds until the process
 * exits.  A problem needing more returns DSCF_ERR_OOM without launching anything (the
 * scratch needed is about (ns + N + 4) * V * sizeof(real) bytes; for example 32^3 with N = 64 in
 * FP64 or 64^3 with N = 48 in FP32 fit).  The first call on a device looks up that device's copy
 * of the array (a one-time set-up per device); make that first call before any stream capture.
 * Every call reuses the same array and overwrites what it needs, so calls whose work overlaps on
 * the GPU (on different streams, or from different threads) race and must be serialised by the
 * caller.  Errors: DSCF_ERR_ARG, DSCF_ERR_OOM, DSCF_ERR_CUDA; dscf_last_error(NULL) has the
 * message.
 */
#define DSCF_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
int dscf_densities_static(const dscf_params* p, int32_t precision, const void* U_in, void* phi_out,
                          void* stream);

/*
 * Learned predictor of the density map (row "learned predictor" of this library; the paper has
 * no such component).  A translation-invariant 3-D network maps the two potentials to the two
 * densities of an A-B melt:
 *   phi_hat_I = phibar_I + y_I - <y_I>,  y = conv3(tanh(conv2(tanh(conv1(U - <U>))))),
 * with circular 5^3 convolutions 2 -> 32 -> 32 -> 2 channels (U - <U> and the output mean removal
 * are per sample and per species, so the input is gauge-free and the output has the exact block
 * masses).  All convolutions run on BF16 tensor cores with FP32 accumulation; FP32 master
 * weights, Adam.  Parameters are one FP32 vector: W1[32][2][125], b1[32], W2[32][32][125], b2[32],
 * W3[2][32][125], b3[2] (kernel offset index (oz+2)*25 + (oy+2)*5 + (ox+2)).
 *
 * A network context works on `batch` samples of an nx x ny x nz periodic grid (nx a multiple of
 * 16); fields are [batch][2][V] float, device memory.  The workspace is caller-owned like the
 * DSCF one.  phibar: host array of the two mean volume fractions.
 */
typedef struct dscf_net dscf_net;
size_t dscf_net_workspace_bytes(int32_t nx, int32_t ny, int32_t nz, int32_t batch);
int dscf_net_init(int32_t nx, int32_t ny, int32_t nz, int32_t batch, uint64_t seed, void* workspace,
                  size_t workspace_bytes, void* stream, dscf_net** out);
int dscf_net_forward(dscf_net* net, const float* U, const double* phibar, float* phi_out);
/* Loss 0.5 mean((phi_hat - phi_target)^2) over all samples, species and sites (returned in *loss,
 * synchronising, if loss != NULL) and its gradient (copied to grads_out if not NULL);
 * phi_work receives phi_hat. */
int dscf_net_gradient(dscf_net* net, const float* U, const float* phi_target, const double* phibar,
                      float* phi_work, double* loss, float* grads_out);
/* One Adam step (lr, beta1 = 0.9, beta2 = 0.999) on the gradient above. */
int dscf_net_train_step(dscf_net* net, const float* U, const float* phi_target, const double* phibar,
                        float* phi_work, float lr, double* loss);
int dscf_net_get_params(dscf_net* net, float* dst);        /* dst: device or host */
int dscf_net_set_params(dscf_net* net, const float* src);  /* resets the Adam moments */
int64_t dscf_net_num_params(void);

/* Tensor-core path of the network's forward convolutions.  path 0 (default): tcgen05 MMAs with
 * operands in shared memory and accumulators in tensor memory where the grid allows it (nx a
 * multiple of 128, ny of 8, sm_103 device), warp-level mma.sync otherwise; path 1: mma.sync
 * always (the backward pass always uses mma.sync).  dscf_net_tensor_path returns 2 when the
 * forward runs on tcgen05, 1 for mma.sync.  dscf_net_status synchronises and returns
 * DSCF_ERR_TIMEOUT if a tcgen05 convolution gave up waiting for its operand copies, its MMAs or
 * its epilogue (every wait is bounded; the output of that call is invalid), then clears the
 * condition. */
int dscf_net_set_tensor_path(dscf_net* net, int32_t path);
int32_t dscf_net_tensor_path(const dscf_net* net);
int dscf_net_status(dscf_net* net);
int dscf_net_free(dscf_net* net);

/* Use a trained network (same grid as the context, batch 1) as the density map inside the
 * self-consistent inversion of dscf_step (the determination of the potentials from the
 * compositions, Sec. 2 after Eq. 17, with the density functional phi[U] of Eq. 2, evaluated by
 * Eqs. 16-17, replaced by the network): one FP32 melt replica only.
 * Every corrector_every-th step (counted from this call, starting with the first) is exact and
 * judges the predictor (this synchronises): after a predictor step by that step's
 * self-consistency error ||phi[U] - phi*||_inf (exact densities at the potential the predictor
 * produced against the composition it inverted), otherwise by the network's own error
 * max |phi_hat[U] - phi[U]| at the exactly inverted potential.  The steps in between use the
 * predictor while the last judgement is <= tol and are exact otherwise (fallback).  ncg_iters is
 * the number of inversion iterations of a predictor step (0: the context's own count); their
 * secant steps are capped at the local-curvature step.  net NULL detaches.  The network context
 * must outlive the attachment.  DSCF_ERR_ARG for an FP64 or batched context, a solvent system,
 * another grid or batch, corrector_every < 1, tol <= 0 or ncg_iters outside 0..32. */
int dscf_set_predictor(dscf_ctx* ctx, dscf_net* net, int32_t corrector_every, double tol, int32_t ncg_iters);
const char* dscf_net_last_error(const dscf_net* net);

#ifdef __cplusplus
}
#endif
#endif /* DSCF_H */
