// Site-parallel kernels of the time step: Fletcher-Reeves bookkeeping, chemical potential
// (Eq. 4), the fused D3Q19 MRT collide-stream with the thermodynamic body force (Eq. 8-14,
// Table 1) and the convection-diffusion update of the compositions (Eq. 3).
//
// Every "flat" kernel runs nblk blocks per replica; block b of replica r covers the sites
// [b*chunk, (b+1)*chunk) and leaves one FP64 partial per reduction in the replica's slot, so
// totals are formed deterministically by the kernels that consume them.
#include "dscf_internal.cuh"

namespace dscf {

#define FLAT_PROLOGUE                                                   \
    const Rep& R = reps[blk2rep[blockIdx.x]];                           \
    const int lb = blockIdx.x - R.blk0;                                 \
    const int V = (int)R.V;                                             \
    const int i0 = lb * R.chunk;                                        \
    const int i1 = min(i0 + R.chunk, V);                                \
    (void)i1;

__device__ __forceinline__ int pslot_gg(int k) { return (k & 1) ? P_GG1 : P_GG0; }

// Site coordinates from the flat index (32-bit unsigned division: the flat index of a replica
// fits in an int).
__device__ __forceinline__ void site_xyz(int i, int nx, int ny, int& x, int& y, int& z) {
    const unsigned q = (unsigned)i / (unsigned)nx;
    x = i - (int)q * nx;
    z = (int)(q / (unsigned)ny);
    y = (int)q - z * ny;
}

// ---------------------------------------------------------------------------------------------
// Normalisation of the quadrature (Eq. 2 prefactor):  phi_I = phi_p/(N Q) q_I,
// phi_S = phi_s exp(-U_S)/<exp(-U_S)>.
// ---------------------------------------------------------------------------------------------
struct Norm {
    double coef, qs, phis;
};
__device__ __forceinline__ Norm norm_of(const Rep& R, double* sh, int net = 0) {
    Norm n;
    if (net) {   // the learned predictor's output is already normalised
        n.coef = 1.0;
        n.qs = 1.0;
        n.phis = 1.0 - R.phi_p;
        return n;
    }
    const double Q = reduce_parts(slot(R, P_Q), R.ntiles, sh) / (double)R.V;
    n.coef = R.phi_p / ((double)R.N * Q);
    n.qs = (R.ns == 3) ? reduce_parts(slot(R, P_ES), R.nblk, sh) / (double)R.V : 1.0;
    n.phis = 1.0 - R.phi_p;
    return n;
}
// phi_I[U] at one site in the field precision (FP64 only in the normalisation constants).
template <typename T>
__device__ __forceinline__ T model_phi(const Rep& R, const Norm& n, int I, int i) {
    if (I < 2) return (T)n.coef * ((const T*)R.q)[(size_t)I * R.V + i];
    return (T)n.phis * ((const T*)R.E)[2 * (size_t)R.V + i] / (T)n.qs;
}

// FP32 fields with V a multiple of 4 are also walked as float4 (4 consecutive sites per thread and
// iteration: 16-byte accesses, every species offset stays 16-byte aligned).
template <typename T>
__device__ __forceinline__ bool flat_vec(int V) {
    if constexpr (sizeof(T) == 4) return (V & 3) == 0;
    return false;
}
__device__ __forceinline__ float4 ld4(const float* p) { return *(const float4*)p; }
// Scale and source of the model density of species I as a float4 stream: coef q_I, or for the
// solvent phis E_S / qs.
__device__ __forceinline__ const float* model_src(const Rep& R, const Norm& n, int I, float& sc) {
    if (I < 2) {
        sc = (float)n.coef;
        return (const float*)R.q + (size_t)I * R.V;
    }
    sc = (float)(n.phis / n.qs);
    return (const float*)R.E + 2 * (size_t)R.V;
}

// Directional derivative at the trial point: h1 = <phi* - phi[U + a1 d], d>.
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_trial(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                        int net) {
    __shared__ double sh[33];
    FLAT_PROLOGUE
    const Norm n = norm_of(R, sh, net);
    const T* phi = (const T*)R.phi;
    const T* d = (const T*)R.d;
    T h1 = T(0);
    if (flat_vec<T>(V)) {
        const int ns = R.ns;
        float sc[3];
        const float* src[3];
#pragma unroll
        for (int I = 0; I < 3; ++I) src[I] = I < ns ? model_src(R, n, I, sc[I]) : nullptr;
        // sites outer, species inner: every load of an iteration is issued together
        _Pragma("unroll 4") for (int i = i0 + 4 * (int)threadIdx.x; i < i1; i += 4 * kFlatThreads) {
#pragma unroll
            for (int I = 0; I < 3; ++I) {
                if (I >= ns) break;
                const size_t o = (size_t)I * V + i;
                const float4 p = ld4((const float*)phi + o), dd = ld4((const float*)d + o), q = ld4(src[I] + i);
                h1 += (T)((p.x - sc[I] * q.x) * dd.x + (p.y - sc[I] * q.y) * dd.y + (p.z - sc[I] * q.z) * dd.z +
                          (p.w - sc[I] * q.w) * dd.w);
            }
        }
    } else {
        for (int I = 0; I < R.ns; ++I)
            _Pragma("unroll 4") for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
                const size_t o = (size_t)I * V + i;
                h1 += (phi[o] - model_phi<T>(R, n, I, i)) * d[o];
            }
    }
    const double t = block_sum((double)h1, sh);
    if (threadIdx.x == 0) slot(R, P_H1)[lb] = t;
    __shared__ int fin;
    if (last_block_of(R, &fin)) {
        const double h1s = reduce_parts_cg(slot(R, P_H1), R.nblk, sh);
        if (threadIdx.x == 0) R.scal[S_H1S] = h1s;
    }
}

// Store phi_m = phi[U] of the committed point; k >= 0 also leaves <g,g> (g = phi* - phi_m) in
// the parity slot of iteration k+1 and max|g|.
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_grad(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                       int k, int net) {
    __shared__ double sh[33];
    FLAT_PROLOGUE
    const Norm n = norm_of(R, sh, net);
    if (lb == 0 && threadIdx.x == 0 && !net) {
        R.scal[S_Q] = n.coef > 0.0 ? R.phi_p / ((double)R.N * n.coef) : 0.0;
        R.scal[S_QS] = n.qs;
    }
    const T* __restrict__ phi = (const T*)R.phi;
    T* __restrict__ pm = (T*)R.phim;   // written only here: loads may move past its stores
    T gg = T(0), gmax = T(0);
    if (flat_vec<T>(V)) {
        const int ns = R.ns;
        float scs[3];
        const float* srcs[3];
#pragma unroll
        for (int I = 0; I < 3; ++I) srcs[I] = I < ns ? model_src(R, n, I, scs[I]) : nullptr;
        // sites outer, species inner: every load of an iteration is issued together
        _Pragma("unroll 4") for (int i = i0 + 4 * (int)threadIdx.x; i < i1; i += 4 * kFlatThreads) {
#pragma unroll
            for (int I = 0; I < 3; ++I) {
                if (I >= ns) break;
                const float sc = scs[I];
                const float* src = srcs[I];
                const size_t o = (size_t)I * V + i;
                const float4 q = ld4(src + i), p = ld4((const float*)phi + o);
                const float4 m = make_float4(sc * q.x, sc * q.y, sc * q.z, sc * q.w);
                *(float4*)((float*)pm + o) = m;
                const float g0 = p.x - m.x, g1 = p.y - m.y, g2 = p.z - m.z, g3 = p.w - m.w;
                gg += (T)(g0 * g0 + g1 * g1 + g2 * g2 + g3 * g3);
                gmax = fmax(gmax, (T)fmaxf(fmaxf(fabsf(g0), fabsf(g1)), fmaxf(fabsf(g2), fabsf(g3))));
            }
        }
    } else {
        for (int I = 0; I < R.ns; ++I)
            _Pragma("unroll 4") for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
                const size_t o = (size_t)I * V + i;
                const T m = model_phi<T>(R, n, I, i);
                pm[o] = m;
                const T g = phi[o] - m;
                gg += g * g;
                gmax = fmax(gmax, fabs(g));
            }
    }
    if (k >= 0) {
        const double t = block_sum((double)gg, sh);
        const double tm = block_max((double)gmax, sh);
        if (threadIdx.x == 0) {
            slot(R, pslot_gg(k + 1))[lb] = t;
            slot(R, P_GMAX)[lb] = tm;
        }
        __shared__ int fin;
        if (last_block_of(R, &fin)) {
            const double ggs = reduce_parts_cg(slot(R, pslot_gg(k + 1)), R.nblk, sh);
            if (threadIdx.x == 0) R.scal[S_GGS0 + ((k + 1) & 1)] = ggs;
        }
    }
}

// Conjugate direction.  mode 0: d = -g (start of an inversion, also <g,g> and max|g|);
// mode 1 (after iteration k): beta = <g_{k+1},g_{k+1}>/<g_k,g_k> (Fletcher-Reeves),
// d = -g + beta d.  Leaves h0 = <g,d> and <d, phi_m d> for the next line search.
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_dir(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                      int mode, int k, int* status) {
    __shared__ double sh[3 * 33];
    FLAT_PROLOGUE
    double beta = 0.0;
    if (mode == 1) {
        // <g,g> of iterations k+1 and k, totalled by the last blocks of their producers
        const double ggn = R.scal[S_GGS0 + ((k + 1) & 1)], ggo = R.scal[S_GGS0 + (k & 1)];
        beta = (ggo > 0.0) ? ggn / ggo : 0.0;
        if (lb == 0) {
            const double gm = reduce_parts_max(slot(R, P_GMAX), R.nblk, sh);
            if (threadIdx.x == 0) {
                R.scal[S_ITER0 + 4 * k + 2] = ggn;
                R.scal[S_ITER0 + 4 * k + 3] = gm;
                if (!isfinite(ggn)) atomicOr(status, (int)ST_NONFINITE);
            }
        }
    }
    const T* __restrict__ phi = (const T*)R.phi;
    const T* __restrict__ pm = (const T*)R.phim;
    T* __restrict__ d = (T*)R.d;
    const T tb = (T)beta;
    T h0 = T(0), cd = T(0), gg = T(0), gmax = T(0);
    if (flat_vec<T>(V)) {
        const float fb = (float)tb;
        _Pragma("unroll 4") for (int i = i0 + 4 * (int)threadIdx.x; i < i1; i += 4 * kFlatThreads) {
            for (int I = 0; I < R.ns; ++I) {
                const size_t o = (size_t)I * V + i;
                const float4 p = ld4((const float*)phi + o), m = ld4((const float*)pm + o);
                float4 dn = make_float4(m.x - p.x, m.y - p.y, m.z - p.z, m.w - p.w);   // -g
                if (mode != 0) {
                    const float4 dd = ld4((const float*)d + o);
                    dn.x += fb * dd.x;
                    dn.y += fb * dd.y;
                    dn.z += fb * dd.z;
                    dn.w += fb * dd.w;
                }
                *(float4*)((float*)d + o) = dn;
                const float g0 = p.x - m.x, g1 = p.y - m.y, g2 = p.z - m.z, g3 = p.w - m.w;
                h0 += (T)(g0 * dn.x + g1 * dn.y + g2 * dn.z + g3 * dn.w);
                cd += (T)(dn.x * m.x * dn.x + dn.y * m.y * dn.y + dn.z * m.z * dn.z + dn.w * m.w * dn.w);
                gg += (T)(g0 * g0 + g1 * g1 + g2 * g2 + g3 * g3);
                gmax = fmax(gmax, (T)fmaxf(fmaxf(fabsf(g0), fabsf(g1)), fmaxf(fabsf(g2), fabsf(g3))));
            }
        }
    } else {
        for (int I = 0; I < R.ns; ++I)
            _Pragma("unroll 4") for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
                const size_t o = (size_t)I * V + i;
                const T g = phi[o] - pm[o];
                const T dn = (mode == 0) ? -g : -g + tb * d[o];
                d[o] = dn;
                h0 += g * dn;
                cd += dn * pm[o] * dn;
                gg += g * g;
                gmax = fmax(gmax, fabs(g));
            }
    }
    if (mode == 0) {
        double t[3] = {(double)h0, (double)cd, (double)gg};
        block_sum_n<3>(t, sh);
        const double tm = block_max((double)gmax, sh);
        if (threadIdx.x == 0) {
            slot(R, P_H0)[lb] = t[0];
            slot(R, P_CD)[lb] = t[1];
            slot(R, P_GG0)[lb] = t[2];
            slot(R, P_GMAX)[lb] = tm;
        }
    } else {
        double t[2] = {(double)h0, (double)cd};
        block_sum_n<2>(t, sh);
        if (threadIdx.x == 0) {
            slot(R, P_H0)[lb] = t[0];
            slot(R, P_CD)[lb] = t[1];
        }
    }
    __shared__ int fin;
    if (last_block_of(R, &fin)) {
        const Parts<2> ps = {slot(R, P_H0), slot(R, P_CD)};
        double t[2];
        reduce_parts_n_cg<2>(ps, R.nblk, t, sh);
        const double gg0 = mode == 0 ? reduce_parts_cg(slot(R, P_GG0), R.nblk, sh) : 0.0;
        if (threadIdx.x == 0) {
            R.scal[S_H0S] = t[0];
            R.scal[S_CDS] = t[1];
            if (mode == 0) R.scal[S_GGS0] = gg0;
        }
    }
}

// Starting point of the inversion from the potentials of the last two steps: once Uprev holds the
// potentials a previous step started from (and they came out of an inversion: scal[S_WARM] = 2),
// U <- 2 U - Uprev, the linear extrapolation in time; in every case Uprev <- the incoming U.  The
// last block advances the history count.
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_extrap(const Rep* __restrict__ reps, const int* __restrict__ blk2rep) {
    FLAT_PROLOGUE
    const bool go = R.scal[S_WARM] >= 2.0;
    T* __restrict__ U = (T*)R.U;
    T* __restrict__ Up = (T*)R.Uprev;
    for (int I = 0; I < R.ns; ++I)
        for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
            const size_t o = (size_t)I * V + i;
            const T u = U[o];
            if (go) U[o] = T(2) * u - Up[o];
            Up[o] = u;
        }
    __shared__ int fin;
    if (last_block_of(R, &fin) && threadIdx.x == 0) R.scal[S_WARM] = go ? 2.0 : R.scal[S_WARM] + 1.0;
}

// sigma[f] at one site, written as the x, y, z passes of the separable 27-point stencil.
template <typename T>
__device__ __forceinline__ T sigma_at(const T* __restrict__ f, int x, int y, int z, int nx, int ny, int nz, T al,
                                      T be) {
    const int xs[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
    const int ys[3] = {y == 0 ? ny - 1 : y - 1, y, y == ny - 1 ? 0 : y + 1};
    const int zs[3] = {z == 0 ? nz - 1 : z - 1, z, z == nz - 1 ? 0 : z + 1};
    T zz[3];
    for (int c = 0; c < 3; ++c) {
        T yy[3];
        for (int b = 0; b < 3; ++b) {
            const int row = nx * (ys[b] + ny * zs[c]);
            yy[b] = be * f[row + xs[1]] + al * (f[row + xs[0]] + f[row + xs[2]]);
        }
        zz[c] = be * yy[1] + al * (yy[0] + yy[2]);
    }
    return be * zz[1] + al * (zz[0] + zz[2]);
}

// Chemical potentials, Eq. 4: mu_I = -U_I + sum_J chi_IJ sigma[phi_J] + kappa (sum_J phi_J - 1).
// Block 0 of each replica also records the end-of-inversion residual.
template <typename T>
__global__ void __launch_bounds__(kFlatThreads, sizeof(T) == 4 ? 3 : 1) k_mu(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                     int K) {
    __shared__ double sh[33];
    FLAT_PROLOGUE
    if (K < 0) K = (int)R.scal[S_NITER];   // iterations the residual stop let run
    if (K >= 1 && lb == 0) {
        const double gg = reduce_parts(slot(R, pslot_gg(K)), R.nblk, sh);
        const double gm = reduce_parts_max(slot(R, P_GMAX), R.nblk, sh);
        if (threadIdx.x == 0) {
            R.scal[S_ITER0 + 4 * (K - 1) + 2] = gg;
            R.scal[S_ITER0 + 4 * (K - 1) + 3] = gm;
        }
    }
    const int nx = R.nx, ny = R.ny, nz = R.nz, ns = R.ns;
    const T al = (T)R.alpha, be = (T)(1.0 - 2.0 * R.alpha);
    const T* phi = (const T*)R.phi;
    const T* U = (const T*)R.U;
    T* mu = (T*)R.mu;
    if constexpr (sizeof(T) == 4) {
        if (nx == 128) {   // whole 128-site rows: one warp per row, four sites per lane
            const int lane = threadIdx.x & 31;
            // x pass of a periodic row held as float4 per lane (neighbours by shuffles)
            auto xpass = [&](float4 v) {
                const float lv = __shfl_sync(0xffffffffu, v.w, (lane + 31) & 31);
                const float rv = __shfl_sync(0xffffffffu, v.x, (lane + 1) & 31);
                return make_float4(be * v.x + al * (lv + v.y), be * v.y + al * (v.x + v.z),
                                   be * v.z + al * (v.y + v.w), be * v.w + al * (v.z + rv));
            };
            auto mix = [&](float4 a, float4 c, float4 d) {   // be c + al (a + d)
                return make_float4(be * c.x + al * (a.x + d.x), be * c.y + al * (a.y + d.y),
                                   be * c.z + al * (a.z + d.z), be * c.w + al * (a.w + d.w));
            };
            // chunks are whole rows (a multiple of 256 sites; nx = 128 divides V)
            for (int rw = i0 / 128 + (int)(threadIdx.x >> 5); rw < i1 / 128; rw += kFlatThreads / 32) {
                const int y = rw % ny, z = rw / ny;
                const int oy0 = 128 * (y == 0 ? ny - 1 : y - 1), oy1 = 128 * y, oy2 = 128 * (y == ny - 1 ? 0 : y + 1);
                const int pz0 = 128 * ny * (z == 0 ? nz - 1 : z - 1), pz1 = 128 * ny * z,
                          pz2 = 128 * ny * (z == nz - 1 ? 0 : z + 1);
                const int i = 128 * rw + 4 * lane;
                // species by species: sigma[phi_J] goes straight into every mu_I
                float4 m[3], tot = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int I = 0; I < 3; ++I) m[I] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
                for (int J = 0; J < ns; ++J) {
                    const float* f = (const float*)phi + (size_t)J * V + 4 * lane;
                    auto plane = [&](int pz) {
                        const float4 a = ld4(f + pz + oy0), c = ld4(f + pz + oy1), d = ld4(f + pz + oy2);
                        if (pz == pz1) tot = make_float4(tot.x + c.x, tot.y + c.y, tot.z + c.z, tot.w + c.w);
                        return mix(xpass(a), xpass(c), xpass(d));
                    };
                    const float4 z0 = plane(pz0), z1 = plane(pz1), z2 = plane(pz2);
                    const float4 sp = mix(z0, z1, z2);
#pragma unroll
                    for (int I = 0; I < 3; ++I) {
                        if (I >= ns) break;
                        const float ch = (float)R.chi[I * 3 + J];
                        m[I].x += ch * sp.x; m[I].y += ch * sp.y; m[I].z += ch * sp.z; m[I].w += ch * sp.w;
                    }
                }
                const float kap = (float)R.kappa;
#pragma unroll
                for (int I = 0; I < 3; ++I) {
                    if (I >= ns) break;
                    const float4 u = ld4((const float*)U + (size_t)I * V + i);
                    float4 o;
                    o.x = -u.x + m[I].x + kap * (tot.x - 1.f);
                    o.y = -u.y + m[I].y + kap * (tot.y - 1.f);
                    o.z = -u.z + m[I].z + kap * (tot.z - 1.f);
                    o.w = -u.w + m[I].w + kap * (tot.w - 1.f);
                    *(float4*)((float*)mu + (size_t)I * V + i) = o;
                }
            }
            return;
        }
    }
    for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
        int x, y, z;
        site_xyz(i, nx, ny, x, y, z);
        T sp[3], tot = T(0);
        for (int J = 0; J < ns; ++J) {
            sp[J] = sigma_at(phi + (size_t)J * V, x, y, z, nx, ny, nz, al, be);
            tot += phi[(size_t)J * V + i];
        }
        for (int I = 0; I < ns; ++I) {
            T m = -U[(size_t)I * V + i];
            for (int J = 0; J < ns; ++J) m += (T)R.chi[I * 3 + J] * sp[J];
            m += (T)R.kappa * (tot - T(1));
            mu[(size_t)I * V + i] = m;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// D3Q19 MRT lattice Boltzmann: pull-scheme fused collide-stream.
// ---------------------------------------------------------------------------------------------
__constant__ signed char kC[19][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1}, {-1, 0, -1},
    {1, 0, -1}, {-1, 0, 1}, {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

// Compile-time D3Q19 velocity components (same order as kC), so unrolled loops fold them.
__host__ __device__ constexpr int lbc(int i, int a) {
    constexpr signed char c[19][3] = {
        {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
        {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1}, {-1, 0, -1},
        {1, 0, -1}, {-1, 0, 1}, {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    return c[i][a];
}

template <typename T>
__device__ __forceinline__ T lbw(int i) {
    return i == 0 ? T(1.0 / 3.0) : (i <= 6 ? T(1.0 / 18.0) : T(1.0 / 36.0));
}

// One collide-stream step at every site, one site per thread.  The stored state is the
// post-collision deviation dn*_i(r) = n*_i(r) - w_i rho0 of the previous step; pulling
// dn*_i(r - c_i) performs the streaming of Eq. 10, then the collision of Eq. 12-13 (noise
// amplitude phi_k = 0) with the force term of Eq. 14 writes the new dn*_i(r) to the other buffer.
//
// Collision in closed form: modes 0-3 are conserved (gamma = 1) with m_0 = 0 and
// m_{1..3} = -f/2 (the half-force velocity of Eq. 9), modes 10-18 have gamma = 0, so
//   n*_i = n_i^eq + Df_i - 3/2 w_i f.c_i + w_i sum_{k=4..9} gamma_k m_k e_ki / b_k,
// where m_4..m_9 are the Table 1 stress modes of the non-equilibrium second moment
// Pi^neq = sum_i (n_i - n_i^eq) c_i c_i and Df_i is Eq. 14 (sum_k w_i m^f_k e_ki/b_k = Df_i).
// The incoming populations only enter through their moments, so each outgoing population is
// formed and stored on its own.  FP32: three CTAs per SM, so that the 19 pulled populations and
// the force inputs stay in registers (at four the compiler spills).
// Ghost modes 10-18 of the D3Q19 basis (Table 1) at velocity c, and their norms
// b_k = sum_i w_i e_ki^2 (only the fluctuating collision needs them: they carry no other signal).
__host__ __device__ constexpr int lb_ghost(int k, int cx, int cy, int cz) {
    const int c2 = cx * cx + cy * cy + cz * cz;
    switch (k) {
        case 10: return (3 * c2 - 5) * cx;
        case 11: return (3 * c2 - 5) * cy;
        case 12: return (3 * c2 - 5) * cz;
        case 13: return (cy * cy - cz * cz) * cx;
        case 14: return (cz * cz - cx * cx) * cy;
        case 15: return (cx * cx - cy * cy) * cz;
        case 16: return 3 * c2 * c2 - 6 * c2 + 1;
        case 17: return (2 * c2 - 3) * (cx * cx - cy * cy);
        default: return (2 * c2 - 3) * (c2 - 3 * cz * cz);
    }
}
__host__ __device__ constexpr double lb_ghost_norm(int k) {
    double b = 0.0;
    for (int i = 0; i < 19; ++i) {
        const int cx = lbc(i, 0), cy = lbc(i, 1), cz = lbc(i, 2);
        const int c2 = cx * cx + cy * cy + cz * cz;
        const double w = c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        const int e = lb_ghost(k, cx, cy, cz);
        b += w * e * e;
    }
    return b;
}

// NOISE: the fluctuating collision of Eq. 13: every non-conserved mode k = 4..18 gains
// phi_k r_k, phi_k = sqrt(rho kT b_k (1 - gamma_k^2) / c_s^2) with the lattice temperature
// kT = dt^2 / Omega; r_k the normals of counters (site, step, 16..19, replica), the step index
// being the device step counter.
template <typename T, bool NOISE>
__global__ void __launch_bounds__(kFlatThreads, sizeof(T) == 4 ? 3 : 2) k_lb(const Rep* __restrict__ reps, int nrep,
                                                        const int* __restrict__ counter, const T* __restrict__ fext) {
    __shared__ double sh[33];
    int r = 0;
    while (r + 1 < nrep && (int)blockIdx.x >= reps[r + 1].lb_blk0) ++r;
    const Rep& R = reps[r];
    const int lbk = blockIdx.x - R.lb_blk0;
    const int V = (int)R.V;
    const int site = lbk * kFlatThreads + threadIdx.x;
    const bool act = site < V;
    const int par = (*counter) & 1;
    const T* src = (const T*)(par ? R.pop1 : R.pop0);
    T* dst = (T*)(par ? R.pop0 : R.pop1);
    const int nx = R.nx, ny = R.ny, nz = R.nz, ns = R.ns;
    const T rho0 = (T)R.rho0, gs = (T)R.gs, gb = (T)R.gb, dt2 = (T)(R.dt * R.dt);
    if (act) {
        const int x = site % nx;
        const int yz = site / nx;
        const int y = yz % ny;
        const int z = yz / ny;
        const int X[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
        const int Y[3] = {y == 0 ? ny - 1 : y - 1, y, y == ny - 1 ? 0 : y + 1};
        const int Z[3] = {z == 0 ? nz - 1 : z - 1, z, z == nz - 1 ? 0 : z + 1};
        // moments of the pulled populations dn*_i(r - c_i) (Eq. 9, deviation form)
        T drho = 0, jx = 0, jy = 0, jz = 0, pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const int cx = lbc(i, 0), cy = lbc(i, 1), cz = lbc(i, 2);
            const int s = X[1 - cx] + nx * (Y[1 - cy] + ny * Z[1 - cz]);
            const T d = src[(size_t)i * V + s];
            drho += d;
            if (cx) { jx += cx * d; pxx += d; }
            if (cy) { jy += cy * d; pyy += d; }
            if (cz) { jz += cz * d; pzz += d; }
            if (cx && cy) pxy += (cx * cy) * d;
            if (cx && cz) pxz += (cx * cz) * d;
            if (cy && cz) pyz += (cy * cz) * d;
        }
        // body force (Eq. 8, central differences), in lattice units dt^2 f
        T fx = 0, fy = 0, fz = 0;
        if (fext) {
            const size_t b3 = 3 * (size_t)R.vbase;
            fx = fext[b3 + site];
            fy = fext[b3 + V + site];
            fz = fext[b3 + 2 * (size_t)V + site];
        } else {
            const T* phi = (const T*)R.phi;
            const T* mu = (const T*)R.mu;
            const int row = nx * (y + ny * z);
            const int sxp = X[2] + row, sxm = X[0] + row;
            const int syp = x + nx * (Y[2] + ny * z), sym = x + nx * (Y[0] + ny * z);
            const int szp = x + nx * (y + ny * Z[2]), szm = x + nx * (y + ny * Z[0]);
            for (int I = 0; I < ns; ++I) {
                const T* m = mu + (size_t)I * V;
                const T ph = phi[(size_t)I * V + site];
                fx -= ph * T(0.5) * (m[sxp] - m[sxm]);
                fy -= ph * T(0.5) * (m[syp] - m[sym]);
                fz -= ph * T(0.5) * (m[szp] - m[szm]);
            }
            fx *= dt2;
            fy *= dt2;
            fz *= dt2;
        }
        const T rho = rho0 + drho;
        jx += T(0.5) * fx;
        jy += T(0.5) * fy;
        jz += T(0.5) * fz;
        const T ux = jx / rho, uy = jy / rho, uz = jz / rho;
        T* uo = (T*)R.u;
        uo[site] = ux;
        uo[V + site] = uy;
        uo[2 * (size_t)V + site] = uz;
        const T usq = ux * ux + uy * uy + uz * uz;
        const T third = T(1.0 / 3.0);
        const T nxx = pxx - rho * ux * ux - drho * third;
        const T nyy = pyy - rho * uy * uy - drho * third;
        const T nzz = pzz - rho * uz * uz - drho * third;
        const T nxy = pxy - rho * ux * uy, nxz = pxz - rho * ux * uz, nyz = pyz - rho * uy * uz;
        const T m4 = nxx + nyy + nzz;
        const T m5 = nxx - nyy;
        const T m6 = m4 - T(3) * nzz;
        // relaxed stress modes divided by their norms b_4 = 2/3, b_5 = 4/9, b_6 = 4/3, b_7..9 = 1/9
        T r4 = gb * m4 * T(1.5);
        T r5 = gs * m5 * T(2.25);
        T r6 = gs * m6 * T(0.75);
        T r7 = gs * nxy * T(9), r8 = gs * nxz * T(9), r9 = gs * nyz * T(9);
        T gk[9];   // ghost modes m*_k / b_k (noise only)
        if constexpr (NOISE) {
            T g[16];
            const unsigned st = (unsigned)(*counter);
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                T n4[4];
                normals4<T>(R.noise_seed, (unsigned)site, st, 16u + (unsigned)cc, (unsigned)R.rep_index, n4);
#pragma unroll
                for (int q = 0; q < 4; ++q) g[4 * cc + q] = n4[q];
            }
            // m*_k / b_k gains phi_k r_k / b_k = sqrt(3 rho kT (1 - gamma_k^2) / b_k) r_k
            const T t3 = T(3) * rho * (T)R.noise_kT;
            const T ab = sqrt(t3 * (T(1) - gb * gb)), as = sqrt(t3 * (T(1) - gs * gs));
            r4 += ab * sqrt(T(1.5)) * g[0];    // b_4 = 2/3
            r5 += as * sqrt(T(2.25)) * g[1];   // b_5 = 4/9
            r6 += as * sqrt(T(0.75)) * g[2];   // b_6 = 4/3
            r7 += as * T(3) * g[3];            // b_7..9 = 1/9
            r8 += as * T(3) * g[4];
            r9 += as * T(3) * g[5];
#pragma unroll
            for (int k = 10; k < 19; ++k) gk[k - 10] = sqrt(t3 / (T)lb_ghost_norm(k)) * g[k - 4];
        }
        // Sigma of Eq. 14
        const T uf = ux * fx + uy * fy + uz * fz;
        const T a1 = T(0.5) * (T(1) + gs), a2 = (T(1) + gb) * third;
        const T sxx = a1 * (T(2) * ux * fx - T(2.0 / 3.0) * uf) + a2 * uf;
        const T syy = a1 * (T(2) * uy * fy - T(2.0 / 3.0) * uf) + a2 * uf;
        const T szz = a1 * (T(2) * uz * fz - T(2.0 / 3.0) * uf) + a2 * uf;
        const T sxy = a1 * (ux * fy + uy * fx), sxz = a1 * (ux * fz + uz * fx), syz = a1 * (uy * fz + uz * fy);
        const T trs3 = (sxx + syy + szz) * third;
        // Every outgoing population is w_i times a quadratic form in c_i: the equilibrium
        // (constant, linear 3 rho u.c, quadratic 9/2 rho (u.c)^2), the forcing (3/2 f.c and
        // 9/2 (c.Sigma.c - tr Sigma / 3)) and the relaxed stress modes (quadratic in c, r_4
        // constant).  Its ten coefficients are formed once per site; per population only the
        // terms with non-zero velocity components remain (c_i in {0, +-1}, known at compile time).
        const T A = drho - T(1.5) * rho * usq - T(4.5) * trs3 - r4;
        const T Bx = T(3) * rho * ux + T(1.5) * fx, By = T(3) * rho * uy + T(1.5) * fy,
                Bz = T(3) * rho * uz + T(1.5) * fz;
        const T Cxx = T(4.5) * (rho * ux * ux + sxx) + r4 + r5 + r6;
        const T Cyy = T(4.5) * (rho * uy * uy + syy) + r4 - r5 + r6;
        const T Czz = T(4.5) * (rho * uz * uz + szz) + r4 - T(2) * r6;
        const T Dxy = T(9) * (rho * ux * uy + sxy) + r7, Dxz = T(9) * (rho * ux * uz + sxz) + r8,
                Dyz = T(9) * (rho * uy * uz + syz) + r9;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const int cx = lbc(i, 0), cy = lbc(i, 1), cz = lbc(i, 2);
            T v = A;
            if (cx) v += (cx > 0 ? Bx : -Bx) + Cxx;
            if (cy) v += (cy > 0 ? By : -By) + Cyy;
            if (cz) v += (cz > 0 ? Bz : -Bz) + Czz;
            if (cx && cy) v += (cx == cy) ? Dxy : -Dxy;
            if (cx && cz) v += (cx == cz) ? Dxz : -Dxz;
            if (cy && cz) v += (cy == cz) ? Dyz : -Dyz;
            if constexpr (NOISE) {
#pragma unroll
                for (int k = 10; k < 19; ++k) {
                    const int e = lb_ghost(k, cx, cy, cz);
                    if (e) v += T(e) * gk[k - 10];
                }
            }
            dst[(size_t)i * V + site] = lbw<T>(i) * v;
        }
    }
}

// LB diagnostics on demand: mass sum_r rho and post-collision momentum sum_r sum_i n*_i c_i of
// the stored populations, max |u_lat|; FP64 per-block partials (flat tiling).
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_lb_diag(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                          const int* __restrict__ counter) {
    __shared__ double sh[33];
    FLAT_PROLOGUE
    const T* cur = (const T*)(((*counter) & 1) ? R.pop1 : R.pop0);
    const T* u = (const T*)R.u;
    T sr = T(0), sx = T(0), sy = T(0), sz = T(0), um = T(0);
    for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            const T d = cur[(size_t)k * V + i];
            sr += d;
            sx += (T)lbc(k, 0) * d;
            sy += (T)lbc(k, 1) * d;
            sz += (T)lbc(k, 2) * d;
        }
        um = fmax(um, fmax(fabs(u[i]), fmax(fabs(u[(size_t)V + i]), fabs(u[2 * (size_t)V + i]))));
    }
    const double a = block_sum((double)sr, sh), bx = block_sum((double)sx, sh), by = block_sum((double)sy, sh),
                 bz = block_sum((double)sz, sh), bm = block_max((double)um, sh);
    if (threadIdx.x == 0) {
        slot(R, P_RHO)[lb] = a;
        slot(R, P_JX)[lb] = bx;
        slot(R, P_JY)[lb] = by;
        slot(R, P_JZ)[lb] = bz;
        slot(R, P_UMAX)[lb] = bm;
    }
}
__global__ void __launch_bounds__(kFlatThreads) k_lb_diag_fin(const Rep* __restrict__ reps, int* status) {
    __shared__ double sh[33];
    const Rep& R = reps[blockIdx.x];
    const double a = reduce_parts(slot(R, P_RHO), R.nblk, sh);
    const double bx = reduce_parts(slot(R, P_JX), R.nblk, sh);
    const double by = reduce_parts(slot(R, P_JY), R.nblk, sh);
    const double bz = reduce_parts(slot(R, P_JZ), R.nblk, sh);
    const double bm = reduce_parts_max(slot(R, P_UMAX), R.nblk, sh);
    if (threadIdx.x == 0) {
        R.scal[S_RHO] = a + R.rho0 * (double)R.V;
        R.scal[S_JX] = bx;
        R.scal[S_JY] = by;
        R.scal[S_JZ] = bz;
        R.scal[S_UMAX] = bm;
        if (!isfinite(a) || !isfinite(bm)) atomicOr(status, (int)ST_NONFINITE);
    }
}

// ---------------------------------------------------------------------------------------------
// Convection-diffusion (Eq. 3): two-step Lax-Wendroff convection, Crank-Nicolson diffusion
// with mu^{n+1} linearised by its local curvature H = diag(1/phi) + kappa 1 1^T, Jacobi
// sweeps, FP64 mass correction.
// ---------------------------------------------------------------------------------------------
struct Nb {
    int n[6];  // +x -x +y -y +z -z
};
__device__ __forceinline__ Nb neighbours(int i, int nx, int ny, int nz) {
    int x, y, z;
    site_xyz(i, nx, ny, x, y, z);
    const int sy = nx, sz = nx * ny;
    Nb b;
    b.n[0] = i + (x == nx - 1 ? 1 - nx : 1);
    b.n[1] = i + (x == 0 ? nx - 1 : -1);
    b.n[2] = i + (y == ny - 1 ? sy - sz : sy);
    b.n[3] = i + (y == 0 ? sz - sy : -sy);
    b.n[4] = i + (z == nz - 1 ? sz - nz * sz : sz);
    b.n[5] = i + (z == 0 ? nz * sz - sz : -sz);
    return b;
}

// Explicit part: rhs_I = -sum_axes [F(i+1/2) - F(i-1/2)] + dt M L(phi; mu^n).  Also stores
// 1/max(phi_I, floor) for the Jacobi sweeps in the Boltzmann-factor buffer, which is free from
// the end of the inversion to the start of the next one.
// NOISE: the composition noise of Eq. 5 joins the explicit part: minus the divergence of a random
// flux on every face, J_a(r) = sqrt(2 M dt / Omega * max(phi_face, 0)) n_a(r), n_a(r) the a-th
// normal of counter (r, step, 1 + I, replica); the step index is the device step counter (the
// step-end kernel of this step has already advanced it).
template <typename T, bool NOISE>
__global__ void __launch_bounds__(kFlatThreads, sizeof(T) == 4 ? (NOISE ? 2 : 4) : 1) k_cd_rhs(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                                        const int* __restrict__ counter) {
    FLAT_PROLOGUE
    const unsigned nstep = NOISE ? (unsigned)(*counter - 1) : 0u;
    const T amp2 = (T)R.noise_amp2;
    const T* phi = (const T*)R.phi;
    const T* mu = (const T*)R.mu;
    const T* u = (const T*)R.u;
    T* rhs = (T*)R.rhs;
    T* inv = (T*)R.E;
    const bool hyd = R.hydro != 0;
    const T dtM = (T)(R.dt * R.M);
    const T fl = (T)R.phi_floor;
    if constexpr (sizeof(T) == 4) {
        const int nx = R.nx, ny = R.ny, nz = R.nz;
        if ((nx & 3) == 0 && nx <= 128 && 128 % nx == 0 && V % 128 == 0) {
            // x rows fill whole warps (chunks are multiples of 256 sites): four consecutive sites
            // per lane, y and z neighbours as float4, x neighbours from the adjacent lanes; the
            // same arithmetic per site as below
            const int lane = threadIdx.x & 31, L = nx >> 2;
            const int lm = (lane % L == 0) ? lane + L - 1 : lane - 1;
            const int lp = (lane % L == L - 1) ? lane - L + 1 : lane + 1;
            const int sy = nx, sz = nx * ny;
            // the field at the x neighbours (-1: q - 1, +1: q + 1) of the four sites
            auto xs = [&](const float4 v, float (&m_)[4], float (&p_)[4]) {
                const float l = __shfl_sync(0xffffffffu, v.w, lm), r = __shfl_sync(0xffffffffu, v.x, lp);
                m_[0] = l; m_[1] = v.x; m_[2] = v.y; m_[3] = v.z;
                p_[0] = v.y; p_[1] = v.z; p_[2] = v.w; p_[3] = r;
            };
            auto arr = [](const float4 v, float (&a)[4]) { a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w; };
            for (int i = i0 + 4 * (int)threadIdx.x; i < i1; i += 4 * kFlatThreads) {
                int x, y, z;
                site_xyz(i, nx, ny, x, y, z);
                const int nyp = i + (y == ny - 1 ? sy - sz : sy), nym = i + (y == 0 ? sz - sy : -sy);
                const int nzp = i + (z == nz - 1 ? sz - nz * sz : sz), nzm = i + (z == 0 ? nz * sz - sz : -sz);
                const int np_[3] = {0, nyp, nzp}, nm_[3] = {0, nym, nzm};
                for (int I = 0; I < R.ns; ++I) {
                    const float* ph = (const float*)phi + (size_t)I * V;
                    const float* m = (const float*)mu + (size_t)I * V;
                    const float4 pc4 = ld4(ph + i), mc4 = ld4(m + i);
                    float pc[4], mc[4], conv[4] = {0.f, 0.f, 0.f, 0.f}, lap[4] = {0.f, 0.f, 0.f, 0.f};
                    arr(pc4, pc);
                    arr(mc4, mc);
                    float nown[4][4], noise[4] = {0.f, 0.f, 0.f, 0.f};
                    if constexpr (NOISE)
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            normals4<float>(R.noise_seed, (unsigned)(i + q), nstep, 1u + (unsigned)I, (unsigned)R.rep_index,
                                            nown[q]);
                    // axis by axis: Courant numbers at the site and its two neighbours, phi and mu
                    // at the neighbours
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        float Ci[4], Cp[4], Cm[4], pp[4], pm[4], mp[4], mm[4];
                        if (hyd) {
                            const float* C = (const float*)u + (size_t)d * V;
                            const float4 c4 = ld4(C + i);
                            arr(c4, Ci);
                            if (d == 0) {
                                xs(c4, Cm, Cp);
                            } else {
                                arr(ld4(C + np_[d]), Cp);
                                arr(ld4(C + nm_[d]), Cm);
                            }
                        } else {
#pragma unroll
                            for (int q = 0; q < 4; ++q) Ci[q] = Cp[q] = Cm[q] = 0.f;
                        }
                        if (d == 0) {
                            xs(pc4, pm, pp);
                            xs(mc4, mm, mp);
                        } else {
                            arr(ld4(ph + np_[d]), pp);
                            arr(ld4(ph + nm_[d]), pm);
                            arr(ld4(m + np_[d]), mp);
                            arr(ld4(m + nm_[d]), mm);
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float hp = 0.5f * (pc[q] + pp[q]) - 0.5f * (Cp[q] * pp[q] - Ci[q] * pc[q]);
                            const float Fp = 0.5f * (Ci[q] + Cp[q]) * hp;
                            const float hm = 0.5f * (pm[q] + pc[q]) - 0.5f * (Ci[q] * pc[q] - Cm[q] * pm[q]);
                            const float Fm = 0.5f * (Cm[q] + Ci[q]) * hm;
                            conv[q] += Fp - Fm;
                            lap[q] += 0.5f * (pc[q] + pp[q]) * (mp[q] - mc[q]) + 0.5f * (pc[q] + pm[q]) * (mm[q] - mc[q]);
                        }
                        if constexpr (NOISE) {
                            // flux through the lower face comes from the neighbour's normals
                            float nlo[4];
                            if (d == 0) {
                                nlo[0] = __shfl_sync(0xffffffffu, nown[3][0], lm);
                                nlo[1] = nown[0][0];
                                nlo[2] = nown[1][0];
                                nlo[3] = nown[2][0];
                            } else {
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    float g[4];
                                    normals4<float>(R.noise_seed, (unsigned)(nm_[d] + q), nstep, 1u + (unsigned)I,
                                                    (unsigned)R.rep_index, g);
                                    nlo[q] = g[d];
                                }
                            }
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                noise[q] += sqrtf((float)amp2 * fmaxf(0.5f * (pm[q] + pc[q]), 0.f)) * nlo[q] -
                                            sqrtf((float)amp2 * fmaxf(0.5f * (pc[q] + pp[q]), 0.f)) * nown[q][d];
                        }
                    }
                    float4 ro, io;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        (&ro.x)[q] = -conv[q] + (float)dtM * lap[q] + noise[q];
                        (&io.x)[q] = 1.f / (pc[q] < (float)fl ? (float)fl : pc[q]);
                    }
                    *(float4*)((float*)rhs + (size_t)I * V + i) = ro;
                    *(float4*)((float*)inv + (size_t)I * V + i) = io;
                }
            }
            return;
        }
    }
    for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
        const Nb b = neighbours(i, R.nx, R.ny, R.nz);
        T Ci[3], Cp[3], Cm[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            Ci[d] = Cp[d] = Cm[d] = T(0);
            if (hyd) {
                const T* C = u + (size_t)d * V;
                Ci[d] = C[i];
                Cp[d] = C[b.n[2 * d]];
                Cm[d] = C[b.n[2 * d + 1]];
            }
        }
        for (int I = 0; I < R.ns; ++I) {
            const T* ph = phi + (size_t)I * V;
            const T* m = mu + (size_t)I * V;
            const T pc = ph[i], mc = m[i];
            T conv = 0, lap = 0, noise = 0;
            T nown[4];
            if constexpr (NOISE)
                normals4<T>(R.noise_seed, (unsigned)i, nstep, 1u + (unsigned)I, (unsigned)R.rep_index, nown);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int ip = b.n[2 * d], im = b.n[2 * d + 1];
                const T pp = ph[ip], pm = ph[im];
                const T hp = T(0.5) * (pc + pp) - T(0.5) * (Cp[d] * pp - Ci[d] * pc);
                const T Fp = T(0.5) * (Ci[d] + Cp[d]) * hp;
                const T hm = T(0.5) * (pm + pc) - T(0.5) * (Ci[d] * pc - Cm[d] * pm);
                const T Fm = T(0.5) * (Cm[d] + Ci[d]) * hm;
                conv += Fp - Fm;
                lap += T(0.5) * (pc + pp) * (m[ip] - mc) + T(0.5) * (pc + pm) * (m[im] - mc);
                if constexpr (NOISE) {
                    T g[4];
                    normals4<T>(R.noise_seed, (unsigned)im, nstep, 1u + (unsigned)I, (unsigned)R.rep_index, g);
                    noise += sqrt(amp2 * fmax(T(0.5) * (pm + pc), T(0))) * g[d] -
                             sqrt(amp2 * fmax(T(0.5) * (pc + pp), T(0))) * nown[d];
                }
            }
            rhs[(size_t)I * V + i] = -conv + dtM * lap + noise;
            inv[(size_t)I * V + i] = T(1) / (pc < fl ? fl : pc);
        }
    }
}

// The Jacobi sweep below for two species with 4 consecutive sites x0..x0+3 of one x row per
// thread: float4 loads at the site and its y and z neighbours, the x neighbours assembled from
// the site's own float4 and the two scalars at x0-1 and x0+4 (periodic).  Same arithmetic per
// site as the scalar sweep.
// SHFL: every warp holds whole x rows (nx divides 128, V a multiple of 128, chunks of whole
// warps), so the x neighbours just outside a thread's four sites come from the adjacent lanes.
template <bool SHFL>
__device__ __forceinline__ void jacobi4(const Rep& R, const float* __restrict__ phi, const float* __restrict__ inv,
                                        const float* __restrict__ rhs, const float* __restrict__ dold,
                                        float* __restrict__ dnew, float c, float kap, int k, int i0, int i1) {
    const int nx = R.nx, ny = R.ny, nz = R.nz;
    const int V = (int)R.V;
    const int sy = nx, sz = nx * ny;
    for (int i = i0 + 4 * (int)threadIdx.x; i < i1; i += 4 * kFlatThreads) {
        int x, y, z;
        site_xyz(i, nx, ny, x, y, z);
        const int nb[4] = {i + (y == ny - 1 ? sy - sz : sy), i + (y == 0 ? sz - sy : -sy),
                           i + (z == nz - 1 ? sz - nz * sz : sz), i + (z == 0 ? nz * sz - sz : -sz)};
        const int ixm = i + (x == 0 ? nx - 1 : -1), ixp = i + (x + 4 == nx ? 4 - nx : 4);
        float4 pc[2];
        float rh[2][4], w[2][4];
#pragma unroll
        for (int I = 0; I < 2; ++I) {
            pc[I] = ld4(phi + (size_t)I * V + i);
#pragma unroll
            for (int q = 0; q < 4; ++q) rh[I][q] = w[I][q] = 0.f;
        }
        // one neighbour direction: values at the neighbour of each of the 4 sites
        auto face = [&](const float (&pn)[2][4], const float (&in_)[2][4], const float (&dn)[2][4]) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float sd = (k > 0) ? dn[0][q] + dn[1][q] : 0.f;
#pragma unroll
                for (int I = 0; I < 2; ++I) {
                    const float pcq = I == 0 ? (&pc[0].x)[q] : (&pc[1].x)[q];
                    const float pf = 0.5f * (pcq + pn[I][q]);
                    w[I][q] += pf;
                    if (k > 0) rh[I][q] += pf * (dn[I][q] * in_[I][q] + kap * sd);
                }
            }
        };
        // y and z neighbours: whole float4 at the neighbouring row
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            float pn[2][4], in_[2][4], dn[2][4];
#pragma unroll
            for (int I = 0; I < 2; ++I) {
                const size_t o = (size_t)I * V + nb[d];
                const float4 a = ld4(phi + o), bi = ld4(inv + o);
                const float4 dd = (k > 0) ? ld4(dold + o) : make_float4(0.f, 0.f, 0.f, 0.f);
                pn[I][0] = a.x; pn[I][1] = a.y; pn[I][2] = a.z; pn[I][3] = a.w;
                in_[I][0] = bi.x; in_[I][1] = bi.y; in_[I][2] = bi.z; in_[I][3] = bi.w;
                dn[I][0] = dd.x; dn[I][1] = dd.y; dn[I][2] = dd.z; dn[I][3] = dd.w;
            }
            face(pn, in_, dn);
        }
        // x neighbours: shifted views of the own float4 plus the scalar just outside it
        {
            float pm_[2][4], im_[2][4], dm_[2][4], pp_[2][4], ip_[2][4], dp_[2][4];
#pragma unroll
            for (int I = 0; I < 2; ++I) {
                const size_t oI = (size_t)I * V;
                const float4 ic = ld4(inv + oI + i);
                const float4 dc = (k > 0) ? ld4(dold + oI + i) : make_float4(0.f, 0.f, 0.f, 0.f);
                float pl, pr, il, ir, dl, dr;
                if constexpr (SHFL) {
                    const int lane = threadIdx.x & 31, L = R.nx >> 2;   // lanes per row
                    const int lm = (lane % L == 0) ? lane + L - 1 : lane - 1;
                    const int lp = (lane % L == L - 1) ? lane - L + 1 : lane + 1;
                    pl = __shfl_sync(0xffffffffu, pc[I].w, lm);
                    pr = __shfl_sync(0xffffffffu, pc[I].x, lp);
                    il = __shfl_sync(0xffffffffu, ic.w, lm);
                    ir = __shfl_sync(0xffffffffu, ic.x, lp);
                    dl = __shfl_sync(0xffffffffu, dc.w, lm);
                    dr = __shfl_sync(0xffffffffu, dc.x, lp);
                } else {
                    pl = phi[oI + ixm]; pr = phi[oI + ixp];
                    il = inv[oI + ixm]; ir = inv[oI + ixp];
                    dl = (k > 0) ? dold[oI + ixm] : 0.f; dr = (k > 0) ? dold[oI + ixp] : 0.f;
                }
                pm_[I][0] = pl; pm_[I][1] = pc[I].x; pm_[I][2] = pc[I].y; pm_[I][3] = pc[I].z;
                pp_[I][0] = pc[I].y; pp_[I][1] = pc[I].z; pp_[I][2] = pc[I].w; pp_[I][3] = pr;
                im_[I][0] = il; im_[I][1] = ic.x; im_[I][2] = ic.y; im_[I][3] = ic.z;
                ip_[I][0] = ic.y; ip_[I][1] = ic.z; ip_[I][2] = ic.w; ip_[I][3] = ir;
                dm_[I][0] = dl; dm_[I][1] = dc.x; dm_[I][2] = dc.y; dm_[I][3] = dc.z;
                dp_[I][0] = dc.y; dp_[I][1] = dc.z; dp_[I][2] = dc.w; dp_[I][3] = dr;
            }
            face(pp_, ip_, dp_);
            face(pm_, im_, dm_);
        }
        // the per-site 2 x 2 block (diagonal plus the rank-one kappa coupling)
        float4 out[2];
        const float4 r0 = ld4(rhs + i), r1 = ld4(rhs + (size_t)V + i);
        const float4 c0 = ld4(inv + i), c1 = ld4(inv + (size_t)V + i);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float rA = (&r0.x)[q] + c * rh[0][q], rB = (&r1.x)[q] + c * rh[1][q];
            const float DA = 1.f + c * w[0][q] * (&c0.x)[q], DB = 1.f + c * w[1][q] * (&c1.x)[q];
            const float AA = c * kap * w[0][q], AB = c * kap * w[1][q];
            const float num = rA / DA + rB / DB, den = 1.f + AA / DA + AB / DB;
            const float sv = num / den;
            (&out[0].x)[q] = (rA - AA * sv) / DA;
            (&out[1].x)[q] = (rB - AB * sv) / DB;
        }
        *(float4*)(dnew + i) = out[0];
        *(float4*)(dnew + (size_t)V + i) = out[1];
    }
}

// One Jacobi sweep k of (I - c L(phi; H .)) delta = rhs, c = dt M / 2; the species block of a
// site is solved exactly (diagonal plus the rank-one kappa coupling).  inv = 1/max(phi, floor)
// from k_cd_rhs.
template <typename T>
__global__ void __launch_bounds__(kFlatThreads, sizeof(T) == 4 ? 4 : 3) k_cd_jacobi(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                            int k) {
    FLAT_PROLOGUE
    const T* phi = (const T*)R.phi;
    const T* inv = (const T*)R.E;
    const T* rhs = (const T*)R.rhs;
    const T* dold = (const T*)((k & 1) ? R.del0 : R.del1);
    T* dnew = (T*)((k & 1) ? R.del1 : R.del0);
    const int ns = R.ns;
    const T c = (T)(0.5 * R.dt * R.M);
    const T kap = (T)R.kappa;
    if constexpr (sizeof(T) == 4) {
        if (ns == 2 && (R.nx & 3) == 0) {   // FP32 melt: 4 consecutive sites of an x row per thread
            // chunks are multiples of 256 sites, so with V a multiple of 128 every warp is whole
            if (R.nx <= 128 && 128 % R.nx == 0 && V % 128 == 0)
                jacobi4<true>(R, (const float*)phi, (const float*)inv, (const float*)rhs, (const float*)dold,
                              (float*)dnew, (float)c, (float)kap, k, i0, i1);
            else
                jacobi4<false>(R, (const float*)phi, (const float*)inv, (const float*)rhs, (const float*)dold,
                               (float*)dnew, (float)c, (float)kap, k, i0, i1);
            return;
        }
    }
    for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
        const Nb b = neighbours(i, R.nx, R.ny, R.nz);
        T rh[3], w[3], phc[3];
#pragma unroll
        for (int I = 0; I < 3; ++I) {
            rh[I] = T(0);
            w[I] = T(0);
            phc[I] = (I < ns) ? phi[(size_t)I * V + i] : T(0);
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int nb = b.n[q];
            // psi at the neighbour from the previous iterate (zero before the first sweep)
            T dl[3], sd = T(0);
#pragma unroll
            for (int J = 0; J < 3; ++J) {
                dl[J] = (J < ns && k > 0) ? dold[(size_t)J * V + nb] : T(0);
                sd += dl[J];
            }
#pragma unroll
            for (int I = 0; I < 3; ++I) {
                if (I < ns) {
                    const T pf = T(0.5) * (phc[I] + phi[(size_t)I * V + nb]);
                    w[I] += pf;                                   // face sum w_I
                    if (k > 0) rh[I] += pf * (dl[I] * inv[(size_t)I * V + nb] + kap * sd);
                }
            }
        }
        T num = T(0), den = T(1), D[3], A[3];
#pragma unroll
        for (int I = 0; I < 3; ++I) {
            if (I < ns) {
                rh[I] = rhs[(size_t)I * V + i] + c * rh[I];
                D[I] = T(1) + c * w[I] * inv[(size_t)I * V + i];
                A[I] = c * kap * w[I];
                num += rh[I] / D[I];
                den += A[I] / D[I];
            }
        }
        const T s = num / den;
#pragma unroll
        for (int I = 0; I < 3; ++I)
            if (I < ns) dnew[(size_t)I * V + i] = (rh[I] - A[I] * s) / D[I];
    }
}

// phi <- phi + delta; FP64 partial sums of each species for the mass correction.
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_cd_finish(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                            int sweeps) {
    __shared__ double sh[33];
    FLAT_PROLOGUE
    T* __restrict__ phi = (T*)R.phi;
    const T* __restrict__ del = (const T*)(((sweeps - 1) & 1) ? R.del1 : R.del0);
    for (int I = 0; I < R.ns; ++I) {
        T acc = T(0);
        if (flat_vec<T>(V)) {
            _Pragma("unroll 2") for (int i = i0 + 4 * (int)threadIdx.x; i < i1; i += 4 * kFlatThreads) {
                const size_t o = (size_t)I * V + i;
                const float4 p = ld4((const float*)phi + o), d = ld4((const float*)del + o);
                const float4 v = make_float4(p.x + d.x, p.y + d.y, p.z + d.z, p.w + d.w);
                *(float4*)((float*)phi + o) = v;
                acc += (T)((v.x + v.y) + (v.z + v.w));
            }
        } else {
            _Pragma("unroll 4") for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
                const size_t o = (size_t)I * V + i;
                const T v = phi[o] + del[o];
                phi[o] = v;
                acc += v;
            }
        }
        const double t = block_sum((double)acc, sh);
        if (threadIdx.x == 0) slot(R, P_MASS0 + I)[lb] = t;
    }
    __shared__ int fin;
    if (last_block_of(R, &fin))
        for (int I = 0; I < R.ns; ++I) {
            const double tot = reduce_parts_cg(slot(R, P_MASS0 + I), R.nblk, sh);
            if (threadIdx.x == 0) R.scal[S_TOT0 + I] = tot;
        }
}

// Shift every species to its prescribed total (FP64); block 0 records the diagnostics.
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_mass_fix(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                           int* status) {
    __shared__ double sh[33];
    FLAT_PROLOGUE
    T* phi = (T*)R.phi;
    for (int I = 0; I < R.ns; ++I) {
        const double tot = R.scal[S_TOT0 + I];   // totalled by the last block of k_cd_finish
        const double shift = (R.mass0[I] - tot) / (double)V;
        if (lb == 0 && threadIdx.x == 0) {
            R.scal[S_DRIFT0 + I] = tot - R.mass0[I];
            R.scal[S_MASS0 + I] = R.mass0[I];
            if (!isfinite(tot)) atomicOr(status, (int)ST_NONFINITE);
        }
        const T ts = (T)shift;
        if (flat_vec<T>(V)) {
            const float fs = (float)ts;
            _Pragma("unroll 2") for (int i = i0 + 4 * (int)threadIdx.x; i < i1; i += 4 * kFlatThreads) {
                float4* p = (float4*)((float*)phi + (size_t)I * V + i);
                const float4 v = *p;
                *p = make_float4(v.x + fs, v.y + fs, v.z + fs, v.w + fs);
            }
        } else {
            _Pragma("unroll 4") for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) phi[(long long)I * V + i] += ts;
        }
    }
}

// Forward map output: phi_ext = phi[U] from the quadrature of the last evaluation.
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_dens_out(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                           T* __restrict__ out) {
    __shared__ double sh[33];
    FLAT_PROLOGUE
    const Norm n = norm_of(R, sh);
    for (int I = 0; I < R.ns; ++I)
        _Pragma("unroll 4") for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads)
            out[R.ext_off + (size_t)I * V + i] = model_phi<T>(R, n, I, i);
}

// Populations in / out: the API exchanges n_i(r) before collision, i.e. the stored
// post-collision deviation streamed: n_i(r) = n*_i(r - c_i).
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_pop_copy(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                           const int* __restrict__ counter, T* __restrict__ ext,
                                                           int dir) {
    FLAT_PROLOGUE
    T* cur = (T*)(((*counter) & 1) ? R.pop1 : R.pop0);
    const long long b19 = 19 * R.vbase;
    const int nx = R.nx, ny = R.ny, nz = R.nz;
    for (int r = i0 + threadIdx.x; r < i1; r += kFlatThreads) {
        const int x = (int)(r % nx);
        const int y = (int)((r / nx) % ny);
        const int z = (int)(r / ((long long)nx * ny));
        for (int i = 0; i < 19; ++i) {
            if (dir == 0) {
                const long long s = wrapi(x - kC[i][0], nx) +
                                    (long long)nx * (wrapi(y - kC[i][1], ny) + (long long)ny * wrapi(z - kC[i][2], nz));
                ext[b19 + (long long)i * V + r] = cur[(long long)i * V + s];
            } else {
                const long long s = wrapi(x + kC[i][0], nx) +
                                    (long long)nx * (wrapi(y + kC[i][1], ny) + (long long)ny * wrapi(z + kC[i][2], nz));
                cur[(long long)i * V + r] = ext[b19 + (long long)i * V + s];
            }
        }
    }
}

// Mass targets: partial sums of the current phi, then one block per replica commits them.
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_mass_parts(const Rep* __restrict__ reps, const int* __restrict__ blk2rep) {
    __shared__ double sh[33];
    FLAT_PROLOGUE
    const T* phi = (const T*)R.phi;
    for (int I = 0; I < R.ns; ++I) {
        T acc = T(0);
        _Pragma("unroll 4") for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) acc += phi[(size_t)I * V + i];
        const double t = block_sum((double)acc, sh);
        if (threadIdx.x == 0) slot(R, P_MASS0 + I)[lb] = t;
    }
}
__global__ void __launch_bounds__(kFlatThreads) k_mass_commit(Rep* reps) {
    __shared__ double sh[33];
    Rep& R = reps[blockIdx.x];
    for (int I = 0; I < R.ns; ++I) {
        const double t = reduce_parts(slot(R, P_MASS0 + I), R.nblk, sh);
        if (threadIdx.x == 0) {
            R.mass0[I] = t;
            R.scal[S_MASS0 + I] = t;
        }
    }
}

__global__ void k_step_end(int* counter) { *counter += 1; }

// ---------------------------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------------------------
template <typename T>
void launch_trial(const Launch& L, int net) {
    k_trial<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, net);
}
template <typename T>
void launch_grad(const Launch& L, int k, int net) {
    k_grad<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, k, net);
}
// Predictor error: max over sites and species of |q - phi_m| (q: predictor output at the current
// U, phi_m: exact phi[U]); one block per replica 0, FP32 fields.
__global__ void __launch_bounds__(kFlatThreads) k_pred_err(const Rep* __restrict__ reps) {
    __shared__ double sh[33];
    const Rep& R = reps[0];
    const float* q = (const float*)R.q;
    const float* pm = (const float*)R.phim;
    const long long V = R.V;
    const long long i0 = (long long)blockIdx.x * R.chunk;
    const long long i1 = min(i0 + (long long)R.chunk, V);
    float m = 0.f;
    for (int I = 0; I < 2; ++I)
        for (long long i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
            const float e = fabsf(q[I * V + i] - pm[I * V + i]);
            m = (e <= m) ? m : (e == e ? e : INFINITY);   // a NaN counts as an infinite error
        }
    const double t = block_max((double)m, sh);
    if (threadIdx.x == 0) slot(R, P_GMAX)[blockIdx.x] = t;
}
__global__ void __launch_bounds__(kFlatThreads) k_pred_err_fin(const Rep* __restrict__ reps) {
    __shared__ double sh[33];
    const Rep& R = reps[0];
    const double t = reduce_parts_max(slot(R, P_GMAX), R.nblk, sh);
    if (threadIdx.x == 0) R.scal[S_PERR] = t;
}
// Free-energy terms and composition sums (Eq. 1 in volume-fraction units, constants dropped):
// per block, sum_r phi_I, sum_r sum_I U_I phi_I and sum_r [1/2 sum_IJ chi_IJ phi_I sigma[phi_J] +
// kappa/2 (sum_I phi_I - 1)^2].
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_obs1(const Rep* __restrict__ reps, const int* __restrict__ blk2rep) {
    __shared__ double sh[33];
    FLAT_PROLOGUE
    const int nx = R.nx, ny = R.ny, nz = R.nz, ns = R.ns;
    const T al = (T)R.alpha, be = (T)(1.0 - 2.0 * R.alpha);
    const T* phi = (const T*)R.phi;
    const T* U = (const T*)R.U;
    T sp[3] = {T(0), T(0), T(0)}, up = T(0), inter = T(0);
    for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
        int x, y, z;
        site_xyz(i, nx, ny, x, y, z);
        T sg[3], ph[3], tot = T(0);
        for (int J = 0; J < ns; ++J) {
            ph[J] = phi[(size_t)J * V + i];
            sg[J] = sigma_at(phi + (size_t)J * V, x, y, z, nx, ny, nz, al, be);
            tot += ph[J];
            sp[J] += ph[J];
            up += U[(size_t)J * V + i] * ph[J];
        }
        T e = T(0);
        for (int I = 0; I < ns; ++I)
            for (int J = 0; J < ns; ++J) e += T(0.5) * (T)R.chi[I * 3 + J] * ph[I] * sg[J];
        e += T(0.5) * (T)R.kappa * (tot - T(1)) * (tot - T(1));
        inter += e;
    }
    const double vals[5] = {(double)sp[0], (double)sp[1], (double)sp[2], (double)up, (double)inter};
    for (int k = 0; k < 5; ++k) {
        const double t = block_sum(vals[k], sh);
        if (threadIdx.x == 0) slot(R, P_OBS0 + k)[lb] = t;
    }
}
// Order parameters of Fig. 1 and Fig. 3 given the species means.
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_obs2(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                      double mA, double mB, double mS) {
    __shared__ double sh[33];
    FLAT_PROLOGUE
    const T* phi = (const T*)R.phi;
    const double m[3] = {mA, mB, mS};
    double s2 = 0.0, seg = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
        for (int I = 0; I < R.ns; ++I) {
            const double d = (double)phi[(size_t)I * V + i] - m[I];
            s2 += d * d;
        }
        seg += fabs((double)phi[i] + (double)phi[(size_t)V + i] - mA - mB);
    }
    const double t2 = block_sum(s2, sh);
    const double ts = block_sum(seg, sh);
    if (threadIdx.x == 0) {
        slot(R, P_OBS0)[lb] = t2;
        slot(R, P_OBS1)[lb] = ts;
    }
}
template <typename T>
void launch_obs1(const Launch& L) {
    k_obs1<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep);
}
template <typename T>
void launch_obs2(const Launch& L, double mA, double mB, double mS) {
    k_obs2<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, mA, mB, mS);
}
template void launch_obs1<float>(const Launch&);
template void launch_obs1<double>(const Launch&);
template void launch_obs2<float>(const Launch&, double, double, double);
template void launch_obs2<double>(const Launch&, double, double, double);

// Minkowski functionals of species I of one replica at a threshold: the body is the union of the
// closed unit cubes of the sites where phi_I > threshold (compared in the field's precision).  Per
// lattice point the kernel counts its cube, the three faces, three edges and the vertex whose lower
// corner it is, each present when one of the 2, 4 or 8 cubes sharing it is in the body; per-block
// integer counts go to partial slots P_OBS0..3 (exact in FP64).
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_minkowski(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                            int replica, int species, T threshold) {
    __shared__ double sh[4 * 33];
    const Rep& R = reps[blk2rep[blockIdx.x]];
    if (R.rep_index != replica) return;
    const int lb = blockIdx.x - R.blk0;
    const int V = (int)R.V;
    const int i0 = lb * R.chunk, i1 = min(i0 + R.chunk, V);
    const int nx = R.nx, ny = R.ny, nz = R.nz;
    const T* f = (const T*)R.phi + (size_t)species * V;
    long long nc = 0, nf = 0, ne = 0, nv = 0;
    for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
        int x, y, z;
        site_xyz(i, nx, ny, x, y, z);
        const int xm = x == 0 ? nx - 1 : x - 1, ym = y == 0 ? ny - 1 : y - 1, zm = z == 0 ? nz - 1 : z - 1;
        const int X[2] = {x, xm}, Y[2] = {y, ym}, Z[2] = {z, zm};
        bool in[2][2][2];   // the cube at (x - dx, y - dy, z - dz)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dz = 0; dz < 2; ++dz) in[dx][dy][dz] = f[X[dx] + nx * (Y[dy] + ny * Z[dz])] > threshold;
        nc += in[0][0][0];
        nf += (in[0][0][0] | in[1][0][0]) + (in[0][0][0] | in[0][1][0]) + (in[0][0][0] | in[0][0][1]);
        ne += (in[0][0][0] | in[1][0][0] | in[0][1][0] | in[1][1][0]) +
              (in[0][0][0] | in[1][0][0] | in[0][0][1] | in[1][0][1]) +
              (in[0][0][0] | in[0][1][0] | in[0][0][1] | in[0][1][1]);
        nv += in[0][0][0] | in[1][0][0] | in[0][1][0] | in[1][1][0] | in[0][0][1] | in[1][0][1] | in[0][1][1] |
              in[1][1][1];
    }
    double t[4] = {(double)nc, (double)nf, (double)ne, (double)nv};
    block_sum_n<4>(t, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) slot(R, P_OBS0 + k)[lb] = t[k];
}

template <typename T>
void launch_minkowski(const Launch& L, int replica, int species, double threshold) {
    k_minkowski<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, replica, species, (T)threshold);
}
template void launch_minkowski<float>(const Launch&, int, int, double);
template void launch_minkowski<double>(const Launch&, int, int, double);

// Trapped solvent, step 1: labels of the complement of {phi_B > threshold}: every complement
// site starts with its own index, body sites with -1 (lab and cnt: 2 V ints of scratch).
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_cc_init(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                          int replica, T threshold, int* __restrict__ lab,
                                                          int* __restrict__ cnt) {
    FLAT_PROLOGUE
    if (R.rep_index != replica) return;
    const T* pb = (const T*)R.phi + (size_t)V;   // species B
    for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
        lab[i] = pb[i] > threshold ? -1 : i;
        cnt[i] = 0;
    }
}
// Step 2, repeated until nothing changes: each complement site takes the smallest label among
// itself and its face neighbours in the complement, then jumps to the label of its label (labels
// only decrease and always name a site of the same component, so concurrent updates are safe);
// at the fixed point every site carries the smallest index of its component.
__global__ void __launch_bounds__(kFlatThreads) k_cc_step(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                          int replica, int* __restrict__ lab, int* __restrict__ changed) {
    FLAT_PROLOGUE
    if (R.rep_index != replica) return;
    const int nx = R.nx, ny = R.ny, nz = R.nz;
    int any = 0;
    for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
        const int l0 = lab[i];
        if (l0 < 0) continue;
        int x, y, z;
        site_xyz(i, nx, ny, x, y, z);
        const int sy = nx, sz = nx * ny;
        const int nb[6] = {i + (x == nx - 1 ? 1 - nx : 1), i + (x == 0 ? nx - 1 : -1),
                           i + (y == ny - 1 ? sy - sz : sy), i + (y == 0 ? sz - sy : -sy),
                           i + (z == nz - 1 ? sz - nz * sz : sz), i + (z == 0 ? nz * sz - sz : -sz)};
        int m = l0;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int ln = lab[nb[k]];
            if (ln >= 0 && ln < m) m = ln;
        }
        const int lj = lab[m];
        if (lj >= 0 && lj < m) m = lj;
        if (m < l0) {
            lab[i] = m;
            any = 1;
        }
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) *changed = 1;
}
// Step 3: component sizes at their roots (the smallest index), then per block: the largest
// component (ties to the smaller root), the number of roots, and the solvent sums.
__global__ void __launch_bounds__(kFlatThreads) k_cc_count(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                           int replica, const int* __restrict__ lab, int* __restrict__ cnt) {
    FLAT_PROLOGUE
    if (R.rep_index != replica) return;
    for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads)
        if (lab[i] >= 0) atomicAdd(&cnt[lab[i]], 1);
}
__global__ void __launch_bounds__(kFlatThreads) k_cc_best(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                          int replica, const int* __restrict__ lab,
                                                          const int* __restrict__ cnt) {
    __shared__ double sh[33];
    __shared__ long long bk[kFlatThreads];
    FLAT_PROLOGUE
    if (R.rep_index != replica) return;
    // key = size * 2^32 + (2^31 - 1 - root): its maximum is the largest component, ties going to
    // the smallest root
    long long best = -1;
    double roots = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads)
        if (lab[i] == i) {
            roots += 1.0;
            const long long key = ((long long)cnt[i] << 32) | (long long)(0x7fffffff - i);
            if (key > best) best = key;
        }
    bk[threadIdx.x] = best;
    __syncthreads();
    for (int o = kFlatThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o && bk[threadIdx.x + o] > bk[threadIdx.x]) bk[threadIdx.x] = bk[threadIdx.x + o];
        __syncthreads();
    }
    const double nr = block_sum(roots, sh);
    if (threadIdx.x == 0) {
        const long long k = bk[0];
        slot(R, P_OBS0)[lb] = k < 0 ? -1.0 : (double)(k >> 32);                          // size
        slot(R, P_OBS1)[lb] = k < 0 ? -1.0 : (double)(0x7fffffff - (int)(k & 0xffffffffLL));   // root
        slot(R, P_OBS4)[lb] = nr;
    }
}
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_cc_solvent(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                             int replica, const int* __restrict__ lab, int bulk) {
    __shared__ double sh[2 * 33];
    FLAT_PROLOGUE
    if (R.rep_index != replica) return;
    const T* ps = (const T*)R.phi + 2 * (size_t)V;
    double tr = 0.0, tot = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
        const double v = (double)ps[i];
        tot += v;
        if (lab[i] >= 0 && lab[i] != bulk) tr += v;
    }
    double t[2] = {tr, tot};
    block_sum_n<2>(t, sh);
    if (threadIdx.x == 0) {
        slot(R, P_OBS2)[lb] = t[0];
        slot(R, P_OBS3)[lb] = t[1];
    }
}

template <typename T>
void launch_cc_init(const Launch& L, int replica, double threshold, int* lab, int* cnt) {
    k_cc_init<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, replica, (T)threshold, lab, cnt);
}
void launch_cc_step(const Launch& L, int replica, int* lab, int* changed) {
    k_cc_step<<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, replica, lab, changed);
}
void launch_cc_count(const Launch& L, int replica, const int* lab, int* cnt) {
    k_cc_count<<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, replica, lab, cnt);
    k_cc_best<<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, replica, lab, cnt);
}
template <typename T>
void launch_cc_solvent(const Launch& L, int replica, const int* lab, int bulk) {
    k_cc_solvent<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, replica, lab, bulk);
}
template void launch_cc_init<float>(const Launch&, int, double, int*, int*);
template void launch_cc_init<double>(const Launch&, int, double, int*, int*);
template void launch_cc_solvent<float>(const Launch&, int, const int*, int);
template void launch_cc_solvent<double>(const Launch&, int, const int*, int);

// One block.  Every replica's residual is reduced in the same fixed order as the kernels that
// record it, so the decision is reproducible; a non-finite residual closes the gate.
// A non-finite <g,g> closes the gate and sets the non-finite status bit.
__global__ void __launch_bounds__(kFlatThreads) k_ncg_gate(const Rep* __restrict__ reps, int nrep, int k, double tol,
                                                           cudaGraphConditionalHandle handle, int* status) {
    __shared__ double sh[33];
    bool open = false, bad = false;
    for (int r = 0; r < nrep; ++r) {
        const Rep& R = reps[r];
        const double gm = reduce_parts_max(slot(R, P_GMAX), R.nblk, sh);
        const double gg = reduce_parts(slot(R, pslot_gg(k)), R.nblk, sh);
        bad = bad || !isfinite(gg);
        open = open || (gm >= tol);
        if (k == 0 && threadIdx.x == 0) {
            R.scal[S_GG0] = gg;
            R.scal[S_GMAX0] = gm;
        }
    }
    open = open && !bad;
    if (threadIdx.x == 0) {
        if (bad) atomicOr(status, (int)ST_NONFINITE);
        for (int r = 0; r < nrep; ++r)
            if (open || k == 0) reps[r].scal[S_NITER] = open ? (double)(k + 1) : 0.0;
        cudaGraphSetConditional(handle, open ? 1u : 0u);
    }
}

void launch_ncg_gate(const Launch& L, int k, double tol, unsigned long long handle) {
    k_ncg_gate<<<1, kFlatThreads, 0, L.stream>>>(L.reps, L.nrep, k, tol, (cudaGraphConditionalHandle)handle,
                                                 L.status);
}

void launch_pred_err(const Launch& L) {
    k_pred_err<<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps);
    k_pred_err_fin<<<1, kFlatThreads, 0, L.stream>>>(L.reps);
}
template <typename T>
void launch_dir(const Launch& L, int mode, int k) {
    k_dir<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, mode, k, L.status);
}
template <typename T>
void launch_extrap(const Launch& L) {
    k_extrap<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep);
}
template <typename T>
void launch_mu(const Launch& L, int K) {
    k_mu<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, K);
}
template <typename T>
void launch_lb(const Launch& L, const void* fext) {
    if (L.noise & 2) k_lb<T, true><<<L.nlb_total, kFlatThreads, 0, L.stream>>>(L.reps, L.nrep, L.counter, (const T*)fext);
    else k_lb<T, false><<<L.nlb_total, kFlatThreads, 0, L.stream>>>(L.reps, L.nrep, L.counter, (const T*)fext);
}
template <typename T>
void launch_cd(const Launch& L, int sweeps) {
    if (L.noise & 1) k_cd_rhs<T, true><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, L.counter);
    else k_cd_rhs<T, false><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, L.counter);
    for (int k = 0; k < sweeps; ++k) k_cd_jacobi<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, k);
    k_cd_finish<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, sweeps);
    k_mass_fix<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, L.status);
}
template <typename T>
void launch_dens_out(const Launch& L, void* phi_ext) {
    k_dens_out<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, (T*)phi_ext);
}
template <typename T>
void launch_pop_copy(const Launch& L, void* ext, int dir) {
    k_pop_copy<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, L.counter, (T*)ext, dir);
}
template <typename T>
void launch_mass_init(const Launch& L, int nrep) {
    k_mass_parts<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep);
    k_mass_commit<<<nrep, kFlatThreads, 0, L.stream>>>(const_cast<Rep*>(L.reps));
}
void launch_step_end(const Launch& L) { k_step_end<<<1, 1, 0, L.stream>>>(L.counter); }
template <typename T>
void launch_lb_diag(const Launch& L) {
    k_lb_diag<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, L.counter);
    k_lb_diag_fin<<<L.nrep, kFlatThreads, 0, L.stream>>>(L.reps, L.status);
}

#define INST(T)                                                        \
    template void launch_trial<T>(const Launch&, int);                 \
    template void launch_grad<T>(const Launch&, int, int);             \
    template void launch_dir<T>(const Launch&, int, int);              \
    template void launch_mu<T>(const Launch&, int);                    \
    template void launch_extrap<T>(const Launch&);                     \
    template void launch_lb<T>(const Launch&, const void*);            \
    template void launch_cd<T>(const Launch&, int);                    \
    template void launch_dens_out<T>(const Launch&, void*);            \
    template void launch_pop_copy<T>(const Launch&, void*, int);       \
    template void launch_mass_init<T>(const Launch&, int);                \
    template void launch_lb_diag<T>(const Launch&);
INST(double)
INST(float)

}  // namespace dscf
