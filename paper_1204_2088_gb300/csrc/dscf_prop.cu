// Green-propagator kernels (Eq. 16-17) and Boltzmann factors.
//
// One launch = one contour step s for every replica whose chain reaches s.  A CTA owns a
// TX x TY column of the lattice and a chunk of zc planes; it streams along z, staging one
// plane (plus a one-site halo in x and y) at a time in shared memory.  The 27-point linkage
// stencil is the tensor product of the 1-D kernel (alpha, 1 - 2 alpha, alpha), so each plane
// gets an x pass and a y pass in shared memory and the z pass combines three consecutive
// planes held in registers.  Inputs of step s are the outputs of step s-1, which at the sizes
// of interest are still resident in the 129 MB L2; the HBM traffic is the write of G_s in the
// forward sweep and its read in the backward sweep.
#include "dscf_internal.cuh"

namespace dscf {

constexpr int TX = 32;
constexpr int TY = 8;

template <typename T>
struct Plane {
    T in[TY + 2][TX + 2];
    T xs[TY + 2][TX];
};

// xy part of the separable stencil on plane z of `src` (nullptr = the constant field 1) at
// this thread's (x, y); all threads of the CTA must call it.
template <typename T>
__device__ __forceinline__ T xy_pass(const T* __restrict__ src, int z, int x0, int y0, int nx, int ny,
                                     int nz, Plane<T>& P, T al, T be) {
    const int tid = threadIdx.x + threadIdx.y * TX;
    const int zz = wrapi(z, nz);
    const long long pofs = (long long)zz * nx * ny;
    for (int i = tid; i < (TY + 2) * (TX + 2); i += TX * TY) {
        const int ly = i / (TX + 2), lx = i - ly * (TX + 2);
        const int gx = wrapi(x0 + lx - 1, nx), gy = wrapi(y0 + ly - 1, ny);
        P.in[ly][lx] = src ? src[pofs + gx + (long long)gy * nx] : T(1);
    }
    __syncthreads();
    for (int row = threadIdx.y; row < TY + 2; row += TY)
        P.xs[row][threadIdx.x] =
            be * P.in[row][threadIdx.x + 1] + al * (P.in[row][threadIdx.x] + P.in[row][threadIdx.x + 2]);
    __syncthreads();
    const T v = be * P.xs[threadIdx.y + 1][threadIdx.x] +
                al * (P.xs[threadIdx.y][threadIdx.x] + P.xs[threadIdx.y + 2][threadIdx.x]);
    __syncthreads();
    return v;
}

// Forward recurrence: G_s = exp(-U_{I_s}) sigma[G_{s-1}], G_0 = 1 (Eq. 17).  At s = N each
// CTA also writes its FP64 partial sum of G_N for Q = V^-1 sum_r G_N(r).
template <typename T>
__global__ void __launch_bounds__(TX* TY) k_prop_fwd(const Rep* __restrict__ reps, const int* __restrict__ tile2rep,
                                                     int s) {
    __shared__ Plane<T> P;
    __shared__ double sh[33];
    const Rep& R = reps[tile2rep[blockIdx.x]];
    const int lt = blockIdx.x - R.tile0;
    const int tx = lt % R.tiles_x, ty = (lt / R.tiles_x) % R.tiles_y, tz = lt / (R.tiles_x * R.tiles_y);
    const int nx = R.nx, ny = R.ny, nz = R.nz;
    const int x0 = tx * TX, y0 = ty * TY, z0 = tz * R.zc, z1 = min(z0 + R.zc, nz);
    const long long V = R.V;
    const T* src = (s == 1) ? nullptr : (const T*)R.G + (long long)(s - 2) * V;
    T* dst = (T*)R.G + (long long)(s - 1) * V;
    const T* E = (const T*)R.E + (s <= R.nA ? 0 : V);
    const T al = (T)R.alpha, be = (T)(1.0 - 2.0 * R.alpha);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool act = (x < nx) && (y < ny);
    const bool lastQ = (s == R.N);
    double qacc = 0.0;
    T pm = xy_pass(src, z0 - 1, x0, y0, nx, ny, nz, P, al, be);
    T p0 = xy_pass(src, z0, x0, y0, nx, ny, nz, P, al, be);
    for (int z = z0; z < z1; ++z) {
        const T pp = xy_pass(src, z + 1, x0, y0, nx, ny, nz, P, al, be);
        if (act) {
            const long long i = x + (long long)nx * (y + (long long)ny * z);
            const T g = E[i] * (be * p0 + al * (pm + pp));
            dst[i] = g;
            if (lastQ) qacc += (double)g;
        }
        pm = p0;
        p0 = pp;
    }
    if (lastQ) {
        const double t = block_sum(qacc, sh);
        if (threadIdx.x == 0 && threadIdx.y == 0) slot(R, P_Q)[lt] = t;
    }
}

// Backward recurrence and contour quadrature (Eq. 16-17), launch j handles s = N - j:
//   sig = sigma[G+_{s+1}] (G+_{N+1} = 1);  q_{I_s} += G_s * sig;  G+_s = exp(-U_{I_s}) * sig.
// G+ only lives in two ping-pong buffers; q_I is (re)started at the first bead of each block.
template <typename T>
__global__ void __launch_bounds__(TX* TY) k_prop_bwd(const Rep* __restrict__ reps, const int* __restrict__ tile2rep,
                                                     int j) {
    __shared__ Plane<T> P;
    const Rep& R = reps[tile2rep[blockIdx.x]];
    const int lt = blockIdx.x - R.tile0;
    const int tx = lt % R.tiles_x, ty = (lt / R.tiles_x) % R.tiles_y, tz = lt / (R.tiles_x * R.tiles_y);
    const int nx = R.nx, ny = R.ny, nz = R.nz;
    const int x0 = tx * TX, y0 = ty * TY, z0 = tz * R.zc, z1 = min(z0 + R.zc, nz);
    const long long V = R.V;
    const int s = R.N - j;
    const T* src = (j == 0) ? nullptr : (const T*)(((j - 1) & 1) ? R.Gp1 : R.Gp0);
    T* dst = (T*)((j & 1) ? R.Gp1 : R.Gp0);
    const T* Gs = (const T*)R.G + (long long)(s - 1) * V;
    const T* E = (const T*)R.E + (s <= R.nA ? 0 : V);
    T* q = (T*)R.q + (s <= R.nA ? 0 : V);
    const bool first = (s == R.N) || (s == R.nA);
    const bool wout = (s > 1);
    const T al = (T)R.alpha, be = (T)(1.0 - 2.0 * R.alpha);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool act = (x < nx) && (y < ny);
    T pm = xy_pass(src, z0 - 1, x0, y0, nx, ny, nz, P, al, be);
    T p0 = xy_pass(src, z0, x0, y0, nx, ny, nz, P, al, be);
    for (int z = z0; z < z1; ++z) {
        const T pp = xy_pass(src, z + 1, x0, y0, nx, ny, nz, P, al, be);
        if (act) {
            const long long i = x + (long long)nx * (y + (long long)ny * z);
            const T sig = be * p0 + al * (pm + pp);
            q[i] = (first ? T(0) : q[i]) + Gs[i] * sig;
            if (wout) dst[i] = E[i] * sig;
        }
        pm = p0;
        p0 = pp;
    }
}

// Boltzmann factors E_I = exp(-U'_I) for the potential U' of the next gradient evaluation:
//   mode 0: U' = U;  mode 1 (trial): U' = U + a1 d with a1 = -<g,d>/<d,phi_m d>;
//   mode 2 (commit): secant step a = a1 (-h0)/(h1 - h0), U <- U + a d, U' = U;
//   mode 3: U' = external potential (forward density map alone).
// Also the FP64 partial sums of exp(-U'_S) for the solvent normalisation.
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_exp(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                      int mode, int k, const T* __restrict__ Uext) {
    __shared__ double sh[33];
    const Rep& R = reps[blk2rep[blockIdx.x]];
    const int lb = blockIdx.x - R.blk0;
    const long long V = R.V;
    const long long i0 = (long long)lb * R.chunk;
    const long long i1 = min(i0 + (long long)R.chunk, V);
    double a = 0.0;
    if (mode == 1 || mode == 2) {
        const double h0 = reduce_parts(slot(R, P_H0), R.nblk, sh);
        const double cd = reduce_parts(slot(R, P_CD), R.nblk, sh);
        const double a1 = (cd > 0.0 && isfinite(h0 / cd)) ? -h0 / cd : 0.0;
        a = a1;
        if (mode == 2) {
            const double h1 = reduce_parts(slot(R, P_H1), R.nblk, sh);
            const double den = h1 - h0;
            a = (den > 0.0) ? a1 * (-h0) / den : a1;
            if (lb == 0 && threadIdx.x == 0) {
                R.scal[S_ITER0 + 4 * k + 0] = a1;
                R.scal[S_ITER0 + 4 * k + 1] = a;
            }
        } else if (k == 0) {
            // start-of-inversion residual (partials written by the direction kernel)
            const double gg = reduce_parts(slot(R, P_GG0), R.nblk, sh);
            const double gm = reduce_parts_max(slot(R, P_GMAX), R.nblk, sh);
            if (lb == 0 && threadIdx.x == 0) {
                R.scal[S_GG0] = gg;
                R.scal[S_GMAX0] = gm;
            }
        }
    }
    const int ns = R.ns;
    T* U = (T*)R.U;
    const T* d = (const T*)R.d;
    T* E = (T*)R.E;
    const T ta = (T)a;
    double es = 0.0;
    for (int I = 0; I < ns; ++I) {
        for (long long i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
            const long long o = (long long)I * V + i;
            T u;
            if (mode == 0) {
                u = U[o];
            } else if (mode == 1) {
                u = U[o] + ta * d[o];
            } else if (mode == 2) {
                u = U[o] + ta * d[o];
                U[o] = u;
            } else {
                u = Uext[R.ext_off + o];
            }
            const T e = bexp(u);
            E[o] = e;
            if (I == 2) es += (double)e;
        }
    }
    if (ns == 3) {
        const double t = block_sum(es, sh);
        if (threadIdx.x == 0) slot(R, P_ES)[lb] = t;
    }
}

template <typename T>
void launch_prop_fwd(const Launch& L, int s, int grid) {
    if (grid <= 0) return;
    k_prop_fwd<T><<<grid, dim3(TX, TY), 0, L.stream>>>(L.reps, L.tile2rep, s);
}
template <typename T>
void launch_prop_bwd(const Launch& L, int j, int grid) {
    if (grid <= 0) return;
    k_prop_bwd<T><<<grid, dim3(TX, TY), 0, L.stream>>>(L.reps, L.tile2rep, j);
}
template <typename T>
void launch_exp(const Launch& L, int mode, int k, const void* Uext) {
    k_exp<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, mode, k, (const T*)Uext);
}

template void launch_prop_fwd<double>(const Launch&, int, int);
template void launch_prop_fwd<float>(const Launch&, int, int);
template void launch_prop_bwd<double>(const Launch&, int, int);
template void launch_prop_bwd<float>(const Launch&, int, int);
template void launch_exp<double>(const Launch&, int, int, const void*);
template void launch_exp<float>(const Launch&, int, int, const void*);

}  // namespace dscf
