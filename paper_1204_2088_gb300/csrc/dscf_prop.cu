// Green-propagator kernels (Eq. 16-17) and Boltzmann factors.
//
// One launch = one contour step s for every replica whose chain reaches s.  A CTA owns ROWS
// lattice rows (plus one halo row on each side, one warp per row) across a range of x and a range
// of zc planes (zc picked per context by the autotuner at initialisation).  Per plane a thread
// applies the x pass of the separable 27-point stencil to its sites, writes them to a
// double-buffered shared row buffer (one barrier per plane), reads the two neighbouring rows for
// the y pass, and combines three consecutive planes in registers for the z pass.
//
// Two row layouts:
//  - whole-row (nx = 32 VEC, VEC = 1, 2, 4): a warp holds an entire periodic x row, VEC
//    consecutive sites per lane; the x pass runs in registers plus two wrap-around shuffles, so no
//    halo is loaded in x and all accesses are VEC-wide vectors;
//  - tiled (any nx): lane L holds column x0 - 1 + L of a 30-column tile, lanes 0 and 31 being the
//    x halo.
//
// Loads are asynchronous: every thread copies its own input sites of plane j + DEPTH - 1 and the
// per-site operands (Boltzmann factor, G_s, q) of the matching output plane into a DEPTH-stage
// shared-memory ring with cp.async, so DEPTH planes per thread are in flight without holding
// registers; a thread only reads ring slots it filled itself, so the ring needs no barrier.  The
// inputs of step s are the outputs of step s-1, still resident in the 129 MB L2 at the sizes of
// interest; the HBM traffic is the write of G_s in the forward sweep and its read in the
// backward sweep.
#include "dscf_internal.cuh"

#include <type_traits>

namespace dscf {

constexpr int NWARP = kPropRows + 2;   // warps per CTA

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
template <int BYTES>
__device__ __forceinline__ void cp_bytes(void* sdst, const void* gsrc) {
    if constexpr (BYTES <= 16) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(sdst)), "l"(gsrc), "n"(BYTES));
    } else {
        cp_bytes<16>(sdst, gsrc);
        cp_bytes<BYTES - 16>((char*)sdst + 16, (const char*)gsrc + 16);
    }
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <typename T, int VEC>
struct alignas(sizeof(T) * VEC <= 16 ? sizeof(T) * VEC : 16) Vec {
    T v[VEC];
};

// Per-launch operands of one replica.
template <typename T>
struct PropOps {
    const T* src;   // nullptr = the constant field 1
    T* dst;
    const T* E;
    const T* Gs;
    T* q;
    bool lastQ, first, wout;
    T al, be;
};

template <typename T, bool BWD>
__device__ __forceinline__ PropOps<T> prop_ops(const Rep& R, int step) {
    PropOps<T> o;
    const size_t V = (size_t)R.V;
    o.Gs = nullptr;
    o.q = nullptr;
    o.lastQ = o.first = false;
    o.wout = true;
    if (!BWD) {
        const int s = step;
        o.src = (s == 1) ? nullptr : (const T*)R.G + (size_t)(s - 2) * V;
        o.dst = (T*)R.G + (size_t)(s - 1) * V;
        o.E = (const T*)R.E + (s <= R.nA ? 0 : V);
        o.lastQ = (s == R.N);
    } else {
        const int s = R.N - step;
        o.src = (step == 0) ? nullptr : (const T*)(((step - 1) & 1) ? R.Gp1 : R.Gp0);
        o.dst = (T*)((step & 1) ? R.Gp1 : R.Gp0);
        o.Gs = (const T*)R.G + (size_t)(s - 1) * V;
        o.E = (const T*)R.E + (s <= R.nA ? 0 : V);
        o.q = (T*)R.q + (s <= R.nA ? 0 : V);
        o.first = (s == R.N) || (s == R.nA);
        o.wout = (s > 1);
    }
    o.al = (T)R.alpha;
    o.be = (T)(1.0 - 2.0 * R.alpha);
    return o;
}

// Shared-memory bytes of one CTA for a replica (host and device agree through this function).
__host__ __device__ constexpr size_t prop_smem(int vec, bool bwd, size_t es) {
    // row buffer (2) + ring stages (input, E, and G, q in the backward sweep)
    return (size_t)(2 + prop_depth(es) * (bwd ? 4 : 2)) * NWARP * 32 * (vec > 0 ? vec : 1) * es;
}

// Whole-row layout: warp w holds row y0 - 1 + w, lane L sites x = VEC L .. VEC L + VEC - 1.
template <typename T, bool BWD, int VEC>
__device__ __forceinline__ double prop_row(const Rep& R, int lt, const PropOps<T>& o, unsigned char* smem) {
    constexpr int D = prop_depth(sizeof(T));
    constexpr int W = 32 * VEC;
    using VT = Vec<T, VEC>;
    T* sX = (T*)smem;                            // [2][NWARP][W]
    T* sRaw = sX + 2 * NWARP * W;                // [D][NWARP][W]
    T* sE = sRaw + D * NWARP * W;                // [D][NWARP][W]
    T* sG = sE + D * NWARP * W;                  // [D][NWARP][W] (backward)
    T* sQ = sG + D * NWARP * W;                  // [D][NWARP][W] (backward)
    const int ty = lt % R.tiles_y, tz = lt / R.tiles_y;
    const int nx = W, ny = R.ny, nz = R.nz;
    const int plane = nx * ny;
    const int y0 = ty * kPropRows;
    const int zb = tz * R.zc, ze = min(zb + R.zc, nz);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int y = y0 - 1 + w;
    const int rowbase = wrapi(y, ny) * nx + VEC * lane;
    const bool outw = (w >= 1) && (w <= kPropRows);
    const bool act = outw && (y < ny);
    const int np = ze - zb + 2;
    const int me = w * W + VEC * lane;           // this thread's slot inside a [NWARP][W] block

    auto issue = [&](int j) {
        if (j < np) {
            const int st = (j % D) * NWARP * W + me;
            if (o.src) {
                int z = zb - 1 + j;
                z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
                cp_bytes<sizeof(VT)>(sRaw + st, o.src + rowbase + z * plane);
            }
            if (act && j >= 2) {
                const int i = rowbase + (zb + j - 2) * plane;
                cp_bytes<sizeof(VT)>(sE + st, o.E + i);
                if (BWD) {
                    cp_bytes<sizeof(VT)>(sG + st, o.Gs + i);
                    if (!o.first) cp_bytes<sizeof(VT)>(sQ + st, o.q + i);
                }
            }
        }
        cp_commit();
    };
#pragma unroll
    for (int j = 0; j < D - 1; ++j) issue(j);

    const T al = o.al, be = o.be;
    double qacc = 0.0;
    T pm[VEC], p0[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) pm[k] = p0[k] = T(0);
    for (int j = 0; j < np; ++j) {
        issue(j + D - 1);
        cp_wait<D - 1>();
        const int st = (j % D) * NWARP * W + me;
        VT v;
        if (o.src) {
            v = *(const VT*)(sRaw + st);
        } else {
#pragma unroll
            for (int k = 0; k < VEC; ++k) v.v[k] = T(1);
        }
        const T lv = __shfl_sync(0xffffffffu, v.v[VEC - 1], (lane + 31) & 31);
        const T rv = __shfl_sync(0xffffffffu, v.v[0], (lane + 1) & 31);
        VT xf;
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            const T l = (k == 0) ? lv : v.v[k - 1];
            const T r = (k == VEC - 1) ? rv : v.v[k + 1];
            xf.v[k] = be * v.v[k] + al * (l + r);
        }
        T* xb = sX + (j & 1) * NWARP * W;
        *(VT*)(xb + me) = xf;
        __syncthreads();
        if (outw) {
            const VT a = *(const VT*)(xb + me - W);
            const VT b = *(const VT*)(xb + me);
            const VT c = *(const VT*)(xb + me + W);
            T yf[VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) yf[k] = be * b.v[k] + al * (a.v[k] + c.v[k]);
            if (j >= 2 && act) {
                const int i = rowbase + (zb + j - 2) * plane;
                const VT e = *(const VT*)(sE + st);
                VT out;
                if (!BWD) {
#pragma unroll
                    for (int k = 0; k < VEC; ++k) {
                        out.v[k] = e.v[k] * (be * p0[k] + al * (pm[k] + yf[k]));
                        if (o.lastQ) qacc += (double)out.v[k];
                    }
                    *(VT*)(o.dst + i) = out;
                } else {
                    const VT g = *(const VT*)(sG + st);
                    VT qv;
                    if (o.first) {
#pragma unroll
                        for (int k = 0; k < VEC; ++k) qv.v[k] = T(0);
                    } else {
                        qv = *(const VT*)(sQ + st);
                    }
#pragma unroll
                    for (int k = 0; k < VEC; ++k) {
                        const T sig = be * p0[k] + al * (pm[k] + yf[k]);
                        qv.v[k] = qv.v[k] + g.v[k] * sig;
                        out.v[k] = e.v[k] * sig;
                    }
                    *(VT*)(o.q + i) = qv;
                    if (o.wout) *(VT*)(o.dst + i) = out;
                }
            }
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                pm[k] = p0[k];
                p0[k] = yf[k];
            }
        }
    }
    cp_wait<0>();
    return qacc;
}

// Tiled layout (any nx): lane L holds column x0 - 1 + L of a 30-column tile.
template <typename T, bool BWD>
__device__ __forceinline__ double prop_tiled(const Rep& R, int lt, const PropOps<T>& o, unsigned char* smem) {
    constexpr int D = prop_depth(sizeof(T));
    constexpr int W = 32;
    T* sX = (T*)smem;
    T* sRaw = sX + 2 * NWARP * W;
    T* sE = sRaw + D * NWARP * W;
    T* sG = sE + D * NWARP * W;
    T* sQ = sG + D * NWARP * W;
    const int txy = R.tiles_x * R.tiles_y;
    const int tz = lt / txy, rem = lt - tz * txy;
    const int ty = rem / R.tiles_x, tx = rem - ty * R.tiles_x;
    const int nx = R.nx, ny = R.ny, nz = R.nz;
    const int plane = nx * ny;
    const int x0 = tx * kPropCols, y0 = ty * kPropRows;
    const int zb = tz * R.zc, ze = min(zb + R.zc, nz);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x = x0 - 1 + lane, y = y0 - 1 + w;
    const int col = wrapi(x, nx) + wrapi(y, ny) * nx;
    const bool act = lane >= 1 && lane <= kPropCols && w >= 1 && w <= kPropRows && x < nx && y < ny;
    const int np = ze - zb + 2;
    const int me = w * W + lane;

    auto issue = [&](int j) {
        if (j < np) {
            const int st = (j % D) * NWARP * W + me;
            if (o.src) {
                int z = zb - 1 + j;
                z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
                cp_bytes<sizeof(T)>(sRaw + st, o.src + col + z * plane);
            }
            if (act && j >= 2) {
                const int i = col + (zb + j - 2) * plane;
                cp_bytes<sizeof(T)>(sE + st, o.E + i);
                if (BWD) {
                    cp_bytes<sizeof(T)>(sG + st, o.Gs + i);
                    if (!o.first) cp_bytes<sizeof(T)>(sQ + st, o.q + i);
                }
            }
        }
        cp_commit();
    };
#pragma unroll
    for (int j = 0; j < D - 1; ++j) issue(j);

    const T al = o.al, be = o.be;
    double qacc = 0.0;
    T pm = T(0), p0 = T(0);
    for (int j = 0; j < np; ++j) {
        issue(j + D - 1);
        cp_wait<D - 1>();
        const int st = (j % D) * NWARP * W + me;
        const T v = o.src ? sRaw[st] : T(1);
        const T l = __shfl_up_sync(0xffffffffu, v, 1);
        const T r = __shfl_down_sync(0xffffffffu, v, 1);
        T* xb = sX + (j & 1) * NWARP * W;
        xb[me] = be * v + al * (l + r);
        __syncthreads();
        if (w >= 1 && w <= kPropRows) {
            const T yf = be * xb[me] + al * (xb[me - W] + xb[me + W]);
            if (j >= 2 && act) {
                const int i = col + (zb + j - 2) * plane;
                const T sig = be * p0 + al * (pm + yf);
                const T e = sE[st];
                if (!BWD) {
                    const T g = e * sig;
                    o.dst[i] = g;
                    if (o.lastQ) qacc += (double)g;
                } else {
                    const T q0 = o.first ? T(0) : sQ[st];
                    o.q[i] = q0 + sG[st] * sig;
                    if (o.wout) o.dst[i] = e * sig;
                }
            }
            pm = p0;
            p0 = yf;
        }
    }
    cp_wait<0>();
    return qacc;
}

// Forward (BWD = false): G_s = exp(-U_{I_s}) sigma[G_{s-1}], G_0 = 1 (Eq. 17); at s = N each CTA
// also writes its FP64 partial sum of G_N for Q = V^-1 sum_r G_N(r).
// Backward (BWD = true), launch j handles s = N - j (Eq. 16-17):
//   sig = sigma[G+_{s+1}] (G+_{N+1} = 1);  q_{I_s} += G_s sig;  G+_s = exp(-U_{I_s}) sig.
// G+ only lives in two ping-pong buffers; q_I is (re)started at the first bead of each block.
template <typename T, bool BWD>
__global__ void __launch_bounds__(32 * NWARP) k_prop(const Rep* __restrict__ reps, const int* __restrict__ tile2rep,
                                                     int step) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double sh[33];
    const Rep& R = reps[tile2rep[blockIdx.x]];
    const int lt = blockIdx.x - R.tile0;
    const PropOps<T> o = prop_ops<T, BWD>(R, step);
    double qacc;
    switch (R.vec) {
        case 4: qacc = prop_row<T, BWD, 4>(R, lt, o, smem); break;
        case 2: qacc = prop_row<T, BWD, 2>(R, lt, o, smem); break;
        case 1: qacc = prop_row<T, BWD, 1>(R, lt, o, smem); break;
        default: qacc = prop_tiled<T, BWD>(R, lt, o, smem); break;
    }
    if (!BWD && o.lastQ) {
        const double t = block_sum(qacc, sh);
        if (threadIdx.x == 0) slot(R, P_Q)[lt] = t;
    }
}

// Rows of 256 sites (8 per lane) in kernels of their own: in the kernels above they would raise
// the register count, and so cut the occupancy, of every other row width.
template <typename T, bool BWD>
__global__ void __launch_bounds__(32 * NWARP) k_prop_w8(const Rep* __restrict__ reps, const int* __restrict__ tile2rep,
                                                        int step) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double sh[33];
    const Rep& R = reps[tile2rep[blockIdx.x]];
    const int lt = blockIdx.x - R.tile0;
    const PropOps<T> o = prop_ops<T, BWD>(R, step);
    const double qacc = prop_row<T, BWD, 8>(R, lt, o, smem);
    if (!BWD && o.lastQ) {
        const double t = block_sum(qacc, sh);
        if (threadIdx.x == 0) slot(R, P_Q)[lt] = t;
    }
}

// ---------------------------------------------------------------------------------------------
// Contour-step fusion (whole-row layout, FP32): one launch advances a group of up to K contour
// steps.  Warp w holds row y0 - K + w (ROWS output rows plus K halo rows on each side); level 0 is
// the group's input field, level k its k-th step.  The CTA streams the planes of its z range
// extended by K on each side through a software pipeline: at pipeline step t it x- and y-filters
// level 0 at plane t, then for k = 1..kg computes level k at plane t - k from the three
// x/y-filtered planes of level k - 1 kept in registers, and x/y-filters it in turn (one barrier
// per level, each level with its own double-buffered row buffer).  The halo shrinks by one row
// and one plane per level, so level kg is exact on the CTA's own rows and planes.
//   forward group g: steps s = gK + k (k = 1..kg); every level's G_s is stored (interior only);
//   backward group g: steps s = N - gK - k + 1; q_{I_s} += G_s sig at every level, and only the
//   last level's G+ is stored.
// Per contour step this reads the previous propagator from L2 once per group instead of once per
// step and saves K - 1 launches per group.
// ---------------------------------------------------------------------------------------------
template <bool BWD, int VEC, int K>
__device__ __forceinline__ double prop_fused_row(const Rep& R, int lt, int g, unsigned char* smem) {
    using T = float;
    constexpr int D = 4;
    constexpr int W = 32 * VEC;
    constexpr int NW = kPropRows + 2 * K;
    using VT = Vec<T, VEC>;
    T* sX = (T*)smem;                            // [K][2][NW][W]
    T* sRaw = sX + K * 2 * NW * W;               // [D][NW][W]
    const int ty = lt % R.tiles_y, tz = lt / R.tiles_y;
    const int ny = R.ny, nz = R.nz, N = R.N, nA = R.nA;
    const int plane = W * ny;
    const size_t V = (size_t)R.V;
    const int y0 = ty * kPropRows;
    const int zb = tz * R.zc, ze = min(zb + R.zc, nz);
    const int zn = ze - zb;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int y = y0 - K + w;
    const int rowbase = wrapi(y, ny) * W + VEC * lane;
    const bool rowout = (w >= K) && (w < K + kPropRows) && (y < ny);
    const int np = zn + 2 * K;                   // level-0 planes zb - K .. ze + K - 1
    const int me = w * W + VEC * lane;
    const T al = (T)R.alpha, be = (T)(1.0 - 2.0 * R.alpha);

    // group geometry
    int kg, sfirst;   // number of levels, contour index of level 1
    const T* src;
    if (!BWD) {
        sfirst = g * K + 1;
        kg = min(K, N - g * K);
        src = (g == 0) ? nullptr : (const T*)R.G + (size_t)(g * K - 1) * V;
    } else {
        sfirst = N - g * K;
        kg = min(K, sfirst);
        src = (g == 0) ? nullptr : (const T*)(((g - 1) & 1) ? R.Gp1 : R.Gp0);
    }
    T* gpout = (T*)((g & 1) ? R.Gp1 : R.Gp0);
    auto level_s = [&](int k) { return BWD ? sfirst - k + 1 : sfirst + k - 1; };
    auto wrapz = [&](int z) { return z < 0 ? z + nz : (z >= nz ? z - nz : z); };

    auto issue = [&](int j) {
        if (j < np && src) {
            cp_bytes<sizeof(VT)>(sRaw + (j % D) * NW * W + me, src + rowbase + wrapz(zb - K + j) * plane);
        }
        cp_commit();
    };
#pragma unroll
    for (int j = 0; j < D - 1; ++j) issue(j);

    // xy[k][m]: x/y-filtered level k at the three most recent planes (m = 0 oldest)
    T xy[K][3][VEC];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int c = 0; c < VEC; ++c) xy[k][m][c] = T(0);
    double qacc = 0.0;

    // x pass of a VEC-vector (periodic row held by the warp) into row buffer `buf`, then barrier,
    // then the y pass of this warp's row.
    auto xyfilter = [&](const VT& v, T* buf, T (&out)[VEC]) {
        const T lv = __shfl_sync(0xffffffffu, v.v[VEC - 1], (lane + 31) & 31);
        const T rv = __shfl_sync(0xffffffffu, v.v[0], (lane + 1) & 31);
        VT xf;
#pragma unroll
        for (int c = 0; c < VEC; ++c) {
            const T l = (c == 0) ? lv : v.v[c - 1];
            const T r = (c == VEC - 1) ? rv : v.v[c + 1];
            xf.v[c] = be * v.v[c] + al * (l + r);
        }
        *(VT*)(buf + me) = xf;
        __syncthreads();
        if (w >= 1 && w < NW - 1) {
            const VT a = *(const VT*)(buf + me - W);
            const VT c = *(const VT*)(buf + me + W);
#pragma unroll
            for (int q = 0; q < VEC; ++q) out[q] = be * xf.v[q] + al * (a.v[q] + c.v[q]);
        } else {
#pragma unroll
            for (int q = 0; q < VEC; ++q) out[q] = T(0);
        }
    };

    for (int t = 0; t < np; ++t) {
        // operands of every level for this pipeline step (level k at plane t - k)
        VT ev[K], gv[K], qv[K];
#pragma unroll
        for (int k = 1; k <= K; ++k) {
            const int p = t - k;
            if (k <= kg && p >= 0 && p < np) {
                const int s = level_s(k);
                const int i = rowbase + wrapz(zb - K + p) * plane;
                ev[k - 1] = *(const VT*)((const T*)R.E + (s <= nA ? 0 : V) + i);
                if (BWD) {
                    gv[k - 1] = *(const VT*)((const T*)R.G + (size_t)(s - 1) * V + i);
                    const bool first = (s == N) || (s == nA);
                    if (!first && rowout && p >= K && p < K + zn) {
                        qv[k - 1] = *(const VT*)((const T*)R.q + (s <= nA ? 0 : V) + i);
                    } else {
#pragma unroll
                        for (int c = 0; c < VEC; ++c) qv[k - 1].v[c] = T(0);
                    }
                }
            }
        }
        // level 0 at plane t
        issue(t + D - 1);
        cp_wait<D - 1>();
        {
            VT v;
            if (src && t < np) {
                v = *(const VT*)(sRaw + (t % D) * NW * W + me);
            } else {
#pragma unroll
                for (int c = 0; c < VEC; ++c) v.v[c] = T(1);
            }
            T out[VEC];
            xyfilter(v, sX + ((0 * 2) + (t & 1)) * NW * W, out);
#pragma unroll
            for (int c = 0; c < VEC; ++c) {
                xy[0][0][c] = xy[0][1][c];
                xy[0][1][c] = xy[0][2][c];
                xy[0][2][c] = out[c];
            }
        }
        // levels 1..K
#pragma unroll
        for (int k = 1; k <= K; ++k) {
            const int p = t - k;                           // plane of level k
            const bool live = (k <= kg);                   // uniform across the CTA
            if (!live) break;
            VT val;
#pragma unroll
            for (int c = 0; c < VEC; ++c)
                val.v[c] = ev[k - 1].v[c] * (be * xy[k - 1][1][c] + al * (xy[k - 1][0][c] + xy[k - 1][2][c]));
            const bool inside = rowout && p >= K && p < K + zn;
            const int s = level_s(k);
            if (p >= 0 && p < np) {
                const int i = rowbase + wrapz(zb - K + p) * plane;
                if (!BWD) {
                    if (inside) {
                        *(VT*)((T*)R.G + (size_t)(s - 1) * V + i) = val;
                        if (s == N) {
#pragma unroll
                            for (int c = 0; c < VEC; ++c) qacc += (double)val.v[c];
                        }
                    }
                } else if (inside) {
                    // val = E sig  ->  q += G_s sig  with sig = val / E recomputed exactly below
                    VT qn;
#pragma unroll
                    for (int c = 0; c < VEC; ++c) {
                        const T sig = be * xy[k - 1][1][c] + al * (xy[k - 1][0][c] + xy[k - 1][2][c]);
                        qn.v[c] = qv[k - 1].v[c] + gv[k - 1].v[c] * sig;
                    }
                    *(VT*)((T*)R.q + (s <= nA ? 0 : V) + i) = qn;
                    if (k == kg && s > 1) *(VT*)(gpout + i) = val;
                }
            }
            if (k < kg) {
                T out[VEC];
                xyfilter(val, sX + ((k * 2) + (t & 1)) * NW * W, out);
#pragma unroll
                for (int c = 0; c < VEC; ++c) {
                    xy[k][0][c] = xy[k][1][c];
                    xy[k][1][c] = xy[k][2][c];
                    xy[k][2][c] = out[c];
                }
            }
        }
    }
    cp_wait<0>();
    return qacc;
}

// Rows of 256 sites: two contour steps per launch (more would spill), in a kernel of their own.
template <bool BWD>
__global__ void __launch_bounds__(32 * (kPropRows + 4)) k_prop_fused_w8(const Rep* __restrict__ reps,
                                                                       const int* __restrict__ tile2rep, int g) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double sh[33];
    const Rep& R = reps[tile2rep[blockIdx.x]];
    const int lt = blockIdx.x - R.tile0;
    const double qacc = prop_fused_row<BWD, 8, 2>(R, lt, g, smem);
    if (!BWD) {
        const bool lastQ = (g * 2 + 2 >= R.N);   // this group reaches s = N
        if (lastQ) {
            const double t = block_sum(qacc, sh);
            if (threadIdx.x == 0) slot(R, P_Q)[lt] = t;
        }
    }
}

template <bool BWD, int K>
__global__ void __launch_bounds__(32 * (kPropRows + 2 * K)) k_prop_fused(const Rep* __restrict__ reps,
                                                                        const int* __restrict__ tile2rep, int g) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double sh[33];
    const Rep& R = reps[tile2rep[blockIdx.x]];
    const int lt = blockIdx.x - R.tile0;
    double qacc;
    switch (R.vec) {
        case 4: qacc = prop_fused_row<BWD, 4, K>(R, lt, g, smem); break;
        case 2: qacc = prop_fused_row<BWD, 2, K>(R, lt, g, smem); break;
        default: qacc = prop_fused_row<BWD, 1, K>(R, lt, g, smem); break;
    }
    if (!BWD) {
        const bool lastQ = (g * K + K >= R.N);   // this group reaches s = N
        if (lastQ) {
            const double t = block_sum(qacc, sh);
            if (threadIdx.x == 0) slot(R, P_Q)[lt] = t;
        }
    }
}

// Boltzmann factors E_I = exp(-U'_I) for the potential U' of the next gradient evaluation:
//   mode 0: U' = U;  mode 1 (trial): U' = U + a1 d with a1 = -<g,d>/<d,phi_m d>;
//   mode 2 (commit): secant step a = a1 (-h0)/(h1 - h0), U <- U + a d, U' = U;
//   mode 3: U' = external potential (forward density map alone).
// Also the FP64 partial sums of exp(-U'_S) for the solvent normalisation.
template <typename T>
__global__ void __launch_bounds__(kFlatThreads) k_exp(const Rep* __restrict__ reps, const int* __restrict__ blk2rep,
                                                      int mode, int k, const T* __restrict__ Uext, int write_u) {
    __shared__ double sh[3 * 33];
    const Rep& R = reps[blk2rep[blockIdx.x]];
    const int lb = blockIdx.x - R.blk0;
    const long long V = R.V;
    const long long i0 = (long long)lb * R.chunk;
    const long long i1 = min(i0 + (long long)R.chunk, V);
    double a = 0.0;
    if (mode == 1 || mode == 2) {
        // totals of the direction and trial kernels' partials, formed by their last blocks
        const double t[3] = {R.scal[S_H0S], R.scal[S_CDS], mode == 2 ? R.scal[S_H1S] : 0.0};
        const double h0 = t[0], cd = t[1];
        const double a1 = (cd > 0.0 && isfinite(h0 / cd)) ? -h0 / cd : 0.0;
        a = a1;
        if (mode == 2) {
            const double h1 = t[2];
            const double den = h1 - h0;
            a = (den > 0.0) ? a1 * (-h0) / den : a1;
            // With the learned predictor the secant is capped at the local-curvature step a1: the
            // exact response is stiffer than the local one (a <= a1), and a network whose response
            // to the tiny trial displacement is below its resolution would otherwise give a
            // near-zero secant denominator and an unbounded step.
            if (write_u && a > a1) a = a1;
            if (lb == 0 && threadIdx.x == 0) {
                R.scal[S_ITER0 + 4 * k + 0] = a1;
                R.scal[S_ITER0 + 4 * k + 1] = a;
            }
        } else if (k == 0 && lb == 0) {
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
    // distinct fields: no store below can change a value loaded from another of them
    T* __restrict__ U = (T*)R.U;
    const T* __restrict__ d = (const T*)R.d;
    T* __restrict__ E = (T*)R.E;
    const T ta = (T)a;
    double es = 0.0;
    bool vec = false;
    if constexpr (sizeof(T) == 4) vec = (V & 3) == 0 && (mode != 3 || (R.ext_off & 3) == 0);
    if (vec) {   // FP32, 4 consecutive sites per thread and iteration (16-byte accesses)
        const float fa = (float)ta;
        float es4 = 0.f;
        const int j0 = (int)i0, j1 = (int)i1;
        constexpr int S = 4 * kFlatThreads;   // sites per block-wide iteration
        // UB iterations of NS species at a time: every load of the batch is issued before the
        // first use (a thread has only a few iterations, so a plain loop would wait for each)
        auto run = [&](auto nsc, auto ubc) {
            constexpr int NS = decltype(nsc)::value, UB = decltype(ubc)::value;
            for (int ib = j0 + 4 * (int)threadIdx.x; ib < j1; ib += UB * S) {
                float4 uu[UB][NS], dv[UB][NS];
#pragma unroll
                for (int it = 0; it < UB; ++it)
#pragma unroll
                    for (int I = 0; I < NS; ++I) {
                        const int i = ib + it * S;
                        if (i < j1) {
                            const size_t o = (size_t)I * V + i;
                            uu[it][I] = (mode == 3) ? *(const float4*)((const float*)Uext + R.ext_off + o)
                                                    : *(const float4*)((const float*)U + o);
                            if (mode == 1 || mode == 2) dv[it][I] = *(const float4*)((const float*)d + o);
                        }
                    }
#pragma unroll
                for (int it = 0; it < UB; ++it)
#pragma unroll
                    for (int I = 0; I < NS; ++I) {
                        const int i = ib + it * S;
                        if (i < j1) {
                            const size_t o = (size_t)I * V + i;
                            float4 u = uu[it][I];
                            if (mode == 1 || mode == 2) {
                                const float4 dd = dv[it][I];
                                u.x += fa * dd.x;
                                u.y += fa * dd.y;
                                u.z += fa * dd.z;
                                u.w += fa * dd.w;
                                if (mode == 2) *(float4*)((float*)U + o) = u;
                            }
                            const float4 e = write_u ? u : make_float4(bexp(u.x), bexp(u.y), bexp(u.z), bexp(u.w));
                            *(float4*)((float*)E + o) = e;
                            if (I == 2) es4 += (e.x + e.y) + (e.z + e.w);
                        }
                    }
            }
        };
        if (ns == 2) run(std::integral_constant<int, 2>{}, std::integral_constant<int, 2>{});
        else run(std::integral_constant<int, 3>{}, std::integral_constant<int, 1>{});
        es += (double)es4;
    }
    for (int I = 0; I < ns && !vec; ++I) {
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
            const T e = write_u ? u : bexp(u);   // write_u: the learned predictor takes U' itself
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
void launch_prop_fwd(const Launch& L, int s, int grid, size_t smem) {
    if (grid <= 0) return;
    if (L.w8) k_prop_w8<T, false><<<grid, 32 * NWARP, smem, L.stream>>>(L.reps, L.tile2rep, s);
    else k_prop<T, false><<<grid, 32 * NWARP, smem, L.stream>>>(L.reps, L.tile2rep, s);
}
template <typename T>
void launch_prop_bwd(const Launch& L, int j, int grid, size_t smem) {
    if (grid <= 0) return;
    if (L.w8) k_prop_w8<T, true><<<grid, 32 * NWARP, smem, L.stream>>>(L.reps, L.tile2rep, j);
    else k_prop<T, true><<<grid, 32 * NWARP, smem, L.stream>>>(L.reps, L.tile2rep, j);
}
size_t prop_fused_smem_bytes(int vec, int K) {
    return (size_t)(K * 2 + 4) * (kPropRows + 2 * K) * 32 * (vec > 0 ? vec : 1) * sizeof(float);
}
int prop_fused_threads(int K) { return 32 * (kPropRows + 2 * K); }
void launch_prop_fused(const Launch& L, bool bwd, int K, int g, int grid, size_t smem) {
    if (grid <= 0) return;
    const int th = prop_fused_threads(K);
    if (L.w8) {   // two steps per launch only (the host never asks for more)
        if (K != 2) return;
        if (bwd) k_prop_fused_w8<true><<<grid, th, smem, L.stream>>>(L.reps, L.tile2rep, g);
        else k_prop_fused_w8<false><<<grid, th, smem, L.stream>>>(L.reps, L.tile2rep, g);
    } else if (K == 2) {
        if (bwd) k_prop_fused<true, 2><<<grid, th, smem, L.stream>>>(L.reps, L.tile2rep, g);
        else k_prop_fused<false, 2><<<grid, th, smem, L.stream>>>(L.reps, L.tile2rep, g);
    } else if (K == 3) {
        if (bwd) k_prop_fused<true, 3><<<grid, th, smem, L.stream>>>(L.reps, L.tile2rep, g);
        else k_prop_fused<false, 3><<<grid, th, smem, L.stream>>>(L.reps, L.tile2rep, g);
    } else {
        if (bwd) k_prop_fused<true, 4><<<grid, th, smem, L.stream>>>(L.reps, L.tile2rep, g);
        else k_prop_fused<false, 4><<<grid, th, smem, L.stream>>>(L.reps, L.tile2rep, g);
    }
}
int prop_fused_set_smem_limit(size_t bytes) {
    cudaError_t e = cudaSuccess;
    const int b = (int)bytes;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prop_fused<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prop_fused<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prop_fused<false, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prop_fused<true, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prop_fused<false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prop_fused<true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    const int b8 = (int)prop_fused_smem_bytes(8, 2);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prop_fused_w8<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b8);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prop_fused_w8<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b8);
    return (int)e;
}

template <typename T>
int prop_set_smem_limit(size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_prop<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_prop<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    const int b8 = (int)prop_smem(8, true, sizeof(T));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prop_w8<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b8);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prop_w8<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b8);
    return (int)e;
}
size_t prop_smem_bytes(int vec, bool bwd, size_t es) { return prop_smem(vec, bwd, es); }
template <typename T>
void launch_exp(const Launch& L, int mode, int k, const void* Uext, int write_u) {
    k_exp<T><<<L.nblk_total, kFlatThreads, 0, L.stream>>>(L.reps, L.blk2rep, mode, k, (const T*)Uext, write_u);
}

template void launch_prop_fwd<double>(const Launch&, int, int, size_t);
template void launch_prop_fwd<float>(const Launch&, int, int, size_t);
template void launch_prop_bwd<double>(const Launch&, int, int, size_t);
template void launch_prop_bwd<float>(const Launch&, int, int, size_t);
template int prop_set_smem_limit<double>(size_t);
template int prop_set_smem_limit<float>(size_t);
template void launch_exp<double>(const Launch&, int, int, const void*, int);
template void launch_exp<float>(const Launch&, int, int, const void*, int);

}  // namespace dscf
