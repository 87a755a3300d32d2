// Persistent contour sweeps (Eq. 16-17) for one replica in the whole-row layout (FP32).
//
// One launch runs a whole forward (or backward) sweep of N contour steps.  The lattice is cut
// into bricks of nx x 8 x BZ sites, one brick per CTA (one CTA per SM for BZ = 16, two for
// BZ = 8; the launch is cooperative, so all CTAs are resident together), one warp per plane of
// the brick.  A warp keeps its plane's x-filtered rows in registers from one contour step to the
// next; per step the CTA only reads the halo rows and planes of its eight y/z neighbours from L2,
// after checking with an acquire load that they have published that step.  Per step:
//   halo rows of the previous step -> x pass -> shared XH (y-halo rows) and ZH (z-halo planes);
//   barrier; each warp y-filters its plane in registers (two halo rows from XH) into shared YS,
//   and one row of a z-halo plane;
//   barrier; z pass (the neighbouring planes from YS) -> sig;
//   forward:  G_s = exp(-U_{I_s}) sig; brick-boundary values stored to the contour stack;
//   backward: q_{I_s} += G_s sig in registers (G_s prefetched a step ahead by bulk copies that
//             complete on an mbarrier, so the halo wait never waits for them),
//             G+_s = exp(-U_{I_s}) sig, boundary values stored to a ping-pong exchange buffer;
//   barrier, release store of the brick's step counter; then the forward interior stores and the
//   x pass of the new values, in registers.
// q is accumulated in registers over a whole block of beads and written once; nothing is
// read-modify-written per step.  Each 1-D pass of the separable stencil is two packed-pair
// operations per two sites (f32x2 add and fma), with the centre weight folded into the Boltzmann
// factors.  Every wait is bounded: on timeout the CTA sets a status bit and a
// global abort flag that makes every other CTA stop waiting, so the launch always finishes.
#include "dscf_internal.cuh"

namespace dscf {

namespace {

constexpr int PBY = 8;                 // brick rows
// Polls of the backward G_s prefetch's mbarrier before giving up.  The copies depend on no other
// CTA, so this bound is fixed and far above any real copy time (a shorter neighbour-wait limit set
// for failure tests must not abandon a copy that is still landing in this CTA's shared memory).
constexpr long long kGsSpinLimit = 1LL << 26;
// Warps per CTA: 16 for bricks of 16 planes (one CTA per SM), 8 for bricks of 8 planes, which
// fit two CTAs per SM so that one brick computes while the other waits on its neighbours.

__device__ __forceinline__ unsigned saddr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp16(void* s, const void* g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr(s)), "l"(g));
}
__device__ __forceinline__ void cpc() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cpw0() { asm volatile("cp.async.wait_group 0;\n" ::); }
__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void bar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void bar_expect(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}
// bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16) completing on bar
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     saddr(dst)),
                 "l"(src), "r"(bytes), "r"(saddr(bar))
                 : "memory");
}
__device__ __forceinline__ bool bar_test(unsigned long long* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred P1;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}\n"
        : "=r"(done)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Packed FP32 pairs (sm_100+ f32x2 arithmetic): two lanes of a float4 per instruction.
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ float4 f4(unsigned long long lo, unsigned long long hi) {
    float4 o;
    upk2(lo, o.x, o.y);
    upk2(hi, o.z, o.w);
    return o;
}

struct PersCtl {
    int* flags;        // one step counter per brick, kFlagStride ints apart
    int* abort;        // set by a CTA that gave up waiting
    int* status;       // device status word
    const int* perm;   // brick of each CTA (NULL: brick = CTA index)
    int limit;         // polls before giving up
};

// Wait until every neighbour brick has published `target`; threads 0..7 poll one neighbour each
// (each counter on its own cache line).  Only the pollers look at the shared abort flag, and only
// every 32 polls, so that the waits of all CTAs do not contend on one line.
__device__ __forceinline__ void wait_nb(const PersCtl& c, const int* nb, int target, bool& aborted) {
    if (threadIdx.x < 8 && !aborted) {
        const int* f = c.flags + (size_t)nb[threadIdx.x] * kFlagStride;
        int spins = 0;
        while (ld_acquire(f) < target) {
            if ((++spins & 31) == 0) {
                if (ld_acquire(c.abort) != 0) {
                    aborted = true;
                    break;
                }
                if (spins > c.limit) {
                    atomicOr(c.status, (int)ST_TIMEOUT);
                    atomicExch(c.abort, 1);
                    aborted = true;
                    break;
                }
            }
            __nanosleep(32);
        }
    }
    __syncthreads();
}

template <int BZ, int NW>
struct PersGeom {
    static constexpr int NH = 2 * (BZ + 2) + 2 * PBY;   // halo rows per step
};

}  // namespace

size_t pers_smem_bytes(int vec, int bz) {
    const size_t W = 32 * (size_t)vec;
    // YS (y-filtered level, planes -1..bz) + XH (x-filtered y-halo rows of the own planes) + ZH
    // (x-filtered z-halo planes, rows -1..8) + halo staging + backward G_s of the brick
    const size_t rows = (size_t)(bz + 2) * PBY + 2 * (size_t)bz + 2 * (PBY + 2) + (2 * (bz + 2) + 2 * PBY) +
                        (size_t)bz * PBY;
    return rows * W * sizeof(float);
}

// Warp w owns plane w of the brick, all PBY rows, four sites of each row per lane; the x-filtered
// rows of the previous level stay in its registers, so the y pass runs in registers (only the two
// y-halo rows of the plane come from shared memory) and only the y-filtered rows go through
// shared memory, for the z pass of the neighbouring planes.  The z-halo planes are y-filtered one
// row per warp.  Brick-boundary values are stored and published first; the rest of the forward
// G_s follows without a fence (the backward G+ interior is never stored: it stays in registers).
template <int BZ, bool BWD, int NW>
__global__ void __launch_bounds__(32 * NW, 16 / NW) k_prop_pers(const Rep* __restrict__ reps, PersCtl ctl) {
    static_assert(NW == BZ, "one warp per plane");
    constexpr int PWARPS = NW, PTHREADS = 32 * NW;
    constexpr int VEC = 4, W = 128;
    using G = PersGeom<BZ, NW>;
    using VT = float4;
    extern __shared__ __align__(16) unsigned char smem[];
    float* YS = (float*)smem;                                  // [BZ+2][PBY][W]
    float* XH = YS + (BZ + 2) * PBY * W;                       // [2][BZ][W]   rows -1 and PBY
    float* ZH = XH + 2 * BZ * W;                               // [2][PBY+2][W] planes -1 and BZ
    float* HS = ZH + 2 * (PBY + 2) * W;                        // [NH][W]
    float* GS = HS + G::NH * W;                                // [BZ][PBY][W] backward G_s
    __shared__ double sh[33];
    __shared__ int nbs[8];
    __shared__ __align__(8) unsigned long long gs_bar;   // backward: completion of the G_s prefetch
    const Rep& R = reps[0];
    const int ny = R.ny, nz = R.nz, N = R.N, nA = R.nA;
    const int plane = W * ny;
    const size_t V = (size_t)R.V;
    const int nby = ny / PBY, nbz = nz / BZ;
    const int b = ctl.perm ? ctl.perm[blockIdx.x] : (int)blockIdx.x;
    const int by = b % nby, bz = b / nby;
    const int y0 = by * PBY, z0 = bz * BZ;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // Each 1-D pass is applied as c + r (a + d) with r = alpha / (1 - 2 alpha), i.e. the
    // stencil's pass divided by its centre weight be = 1 - 2 alpha; the three passes then give
    // sigma / be^3, and be^3 is folded into the Boltzmann factors (and into q at its write-out).
    const double be_d = 1.0 - 2.0 * R.alpha;
    const float rr = (float)(R.alpha / be_d), be3 = (float)(be_d * be_d * be_d);
    const unsigned long long rr2 = pk2(rr, rr), be32 = pk2(be3, be3);
    if (threadIdx.x < 8) {
        const int k = threadIdx.x < 4 ? threadIdx.x : threadIdx.x + 1;   // skip the centre
        const int dy = k % 3 - 1, dz = k / 3 - 1;
        nbs[threadIdx.x] = (by + dy + nby) % nby + nby * ((bz + dz + nbz) % nbz);
    }
    // halo row h -> (row r, plane pl) of the brick's frame, r in -1..PBY, pl in -1..BZ
    auto halo_rp = [&](int h, int& r, int& pl) {
        if (h < 2 * (BZ + 2)) { r = (h < BZ + 2) ? -1 : PBY; pl = h % (BZ + 2) - 1; }
        else { const int h2 = h - 2 * (BZ + 2); pl = (h2 < PBY) ? -1 : BZ; r = h2 % PBY; }
    };
    // where the x-filtered halo row lives: a y-halo row of an own plane, or a z-halo plane row
    auto halo_dst = [&](int r, int pl) -> float* {
        if (pl >= 0 && pl < BZ) return XH + ((r < 0 ? 0 : 1) * BZ + pl) * W;
        return ZH + ((pl < 0 ? 0 : 1) * (PBY + 2) + (r + 1)) * W;
    };
    __shared__ int hoff[2 * (BZ + 2) + 2 * PBY];   // global row offsets of the halo rows
    for (int h = threadIdx.x; h < G::NH; h += PTHREADS) {
        int r, pl;
        halo_rp(h, r, pl);
        const int y = (y0 + r + ny) % ny, z = (z0 + pl + nz) % nz;
        hoff[h] = z * plane + y * W;
    }
    const int c0 = ctl.flags[(size_t)b * kFlagStride];   // step counters of all bricks are equal at launch
    bool aborted = ld_acquire(ctl.abort) != 0;

    auto xpass = [&](VT v) -> VT {      // x pass of a periodic row held by the warp: v + r (left + right)
        const float lv = __shfl_sync(0xffffffffu, v.w, (lane + 31) & 31);
        const float rv = __shfl_sync(0xffffffffu, v.x, (lane + 1) & 31);
        const unsigned long long mid = pk2(v.y, v.z);
        const unsigned long long tlo = add2(pk2(lv, v.x), mid), thi = add2(mid, pk2(v.w, rv));
        return f4(fma2(rr2, tlo, pk2(v.x, v.y)), fma2(rr2, thi, pk2(v.z, v.w)));
    };
    auto mix = [&](VT a, VT c, VT d) -> VT {   // c + r (a + d)
        const unsigned long long tlo = add2(pk2(a.x, a.y), pk2(d.x, d.y));
        const unsigned long long thi = add2(pk2(a.z, a.w), pk2(d.z, d.w));
        return f4(fma2(rr2, tlo, pk2(c.x, c.y)), fma2(rr2, thi, pk2(c.z, c.w)));
    };
    auto ys = [&](int pl, int r) { return YS + ((pl + 1) * PBY + r) * W + VEC * lane; };
    const bool face_plane = (w == 0 || w == BZ - 1);
    auto is_boundary = [&](int r) { return face_plane || r == 0 || r == PBY - 1; };
    // own plane never wraps: offset of (row r, plane w) is own0 + r * W
    const size_t own0 = (size_t)(z0 + w) * plane + (size_t)y0 * W + VEC * lane;

    VT e[PBY];
    auto load_e = [&](int species) {
        const float* E = (const float*)R.E + (size_t)species * V;
#pragma unroll
        for (int r = 0; r < PBY; ++r) {
            const VT v = *(const VT*)(E + own0 + (size_t)r * W);
            e[r] = f4(mul2(be32, pk2(v.x, v.y)), mul2(be32, pk2(v.z, v.w)));
        }
    };
    auto q_out = [&](VT v) -> VT { return f4(mul2(be32, pk2(v.x, v.y)), mul2(be32, pk2(v.z, v.w))); };
    // backward: G_s of the brick into GS, issued by thread 0 as one bulk copy per plane (the
    // plane's PBY rows are contiguous in memory and in GS); the copies complete on gs_bar
    unsigned gs_phase = 0;
    bool gs_pending = false, gs_dead = false;
    auto prefetch_gs = [&](int s) {
        if (gs_dead) return;   // a copy that never completed: issue no more
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // after the generic reads of GS
            const float* Gs = (const float*)R.G + (size_t)(s - 1) * V + (size_t)z0 * plane + (size_t)y0 * W;
            bar_expect(&gs_bar, (unsigned)(BZ * PBY * W * sizeof(float)));
            for (int pl = 0; pl < BZ; ++pl)
                bulk_g2s(GS + pl * PBY * W, Gs + (size_t)pl * plane, (unsigned)(PBY * W * sizeof(float)), &gs_bar);
        }
        gs_pending = true;
    };
    // bounded wait for the pending prefetch; on timeout the CTA reports it, raises the abort and
    // stops prefetching (the copy stays pending for the last wait at the end of the sweep)
    auto wait_gs = [&]() {
        if (!gs_pending || gs_dead) return;
        for (long long spins = 0; !bar_test(&gs_bar, gs_phase); ++spins) {
            if (spins > kGsSpinLimit) {
                atomicOr(ctl.status, (int)ST_TIMEOUT);
                atomicExch(ctl.abort, 1);
                aborted = true;
                gs_dead = true;
                return;
            }
        }
        gs_phase ^= 1u;
        gs_pending = false;
    };

    // the first input (G_0 = 1, or G+_{N+1} = 1): its x pass is 1 + 2 r everywhere
    const float one = 1.0f + 2.0f * rr;
    VT xf[PBY];
#pragma unroll
    for (int r = 0; r < PBY; ++r) xf[r] = make_float4(one, one, one, one);
    for (int i = threadIdx.x; i < (2 * BZ + 2 * (PBY + 2)) * W; i += PTHREADS) XH[i] = one;   // XH and ZH
    VT qacc[BWD ? PBY : 1];
#pragma unroll
    for (int r = 0; r < (BWD ? PBY : 1); ++r) qacc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    float qsum = 0.f;
    int species = BWD ? (N <= nA ? 0 : 1) : (1 <= nA ? 0 : 1);
    load_e(species);
    if (BWD) {
        if (threadIdx.x == 0) bar_init(&gs_bar);
        __syncthreads();
        prefetch_gs(N);
    }
    __syncthreads();

    for (int j = 0; j < N; ++j) {
        const int s = BWD ? N - j : j + 1;
        const int sp = (s <= nA) ? 0 : 1;
        if (sp != species) {
            if (BWD) {   // leaving the B block: its quadrature is complete
                float* q = (float*)R.q + (size_t)species * V;
#pragma unroll
                for (int r = 0; r < PBY; ++r) {
                    *(VT*)(q + own0 + (size_t)r * W) = q_out(qacc[r]);
                    qacc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            species = sp;
            load_e(species);
        }
        // halo of the previous step, x-filtered into XH / ZH
        if (j > 0) {
            wait_nb(ctl, nbs, c0 + j, aborted);
            const float* src = BWD ? (const float*)(((j - 1) & 1) ? R.Gp1 : R.Gp0)
                                   : (const float*)R.G + (size_t)(s - 2) * V;
            for (int h = w; h < G::NH; h += PWARPS) cp16(HS + h * W + VEC * lane, src + hoff[h] + VEC * lane);
            cpc();
            cpw0();
            for (int h = w; h < G::NH; h += PWARPS) {
                int r, pl;
                halo_rp(h, r, pl);
                *(VT*)(halo_dst(r, pl) + VEC * lane) = xpass(*(const VT*)(HS + h * W + VEC * lane));
            }
        }
        __syncthreads();
        // y pass of the own plane in registers (its two y-halo rows from XH), into YS
        {
            const VT top = *(const VT*)(XH + w * W + VEC * lane);          // row -1
            const VT bot = *(const VT*)(XH + (BZ + w) * W + VEC * lane);   // row PBY
            VT prev = top;
#pragma unroll
            for (int r = 0; r < PBY; ++r) {
                const VT nxt = (r + 1 < PBY) ? xf[r + 1] : bot;
                const VT yv = mix(prev, xf[r], nxt);
                prev = xf[r];
                xf[r] = yv;   // xf now holds the y-filtered rows
                *(VT*)ys(w, r) = yv;
            }
        }
        // y pass of the z-halo planes, one row per warp (PBY rows of each of the two planes)
        for (int t = w; t < 2 * PBY; t += PWARPS) {
            const int side = t / PBY, r = t % PBY;
            const float* zr = ZH + (side * (PBY + 2) + r + 1) * W + VEC * lane;
            *(VT*)ys(side ? BZ : -1, r) = mix(*(const VT*)(zr - W), *(const VT*)zr, *(const VT*)(zr + W));
        }
        __syncthreads();
        // z pass and step output
        float* dst = BWD ? (float*)((j & 1) ? R.Gp1 : R.Gp0) : (float*)R.G + (size_t)(s - 1) * V;
        if (BWD) wait_gs();
        VT out[PBY];
#pragma unroll
        for (int r = 0; r < PBY; ++r) {
            const VT a = *(const VT*)ys(w - 1, r), d = *(const VT*)ys(w + 1, r);
            const unsigned long long sglo = fma2(rr2, add2(pk2(a.x, a.y), pk2(d.x, d.y)), pk2(xf[r].x, xf[r].y));
            const unsigned long long sghi = fma2(rr2, add2(pk2(a.z, a.w), pk2(d.z, d.w)), pk2(xf[r].z, xf[r].w));
            out[r] = f4(mul2(pk2(e[r].x, e[r].y), sglo), mul2(pk2(e[r].z, e[r].w), sghi));
            if (BWD) {
                const VT g = *(const VT*)(GS + (w * PBY + r) * W + VEC * lane);
                qacc[r] = f4(fma2(pk2(g.x, g.y), sglo, pk2(qacc[r].x, qacc[r].y)),
                             fma2(pk2(g.z, g.w), sghi, pk2(qacc[r].z, qacc[r].w)));
            } else if (s == N) {
                qsum += (out[r].x + out[r].y) + (out[r].z + out[r].w);
            }
            if (is_boundary(r) && (!BWD || s > 1)) *(VT*)(dst + own0 + (size_t)r * W) = out[r];
        }
        // publish the boundary of this step: the CTA barrier orders every thread's boundary stores
        // before thread 0's release store, and release is cumulative, so a CTA whose acquire load
        // reads the new counter sees them.  The barrier also ends every warp's reads of YS, XH
        // and ZH for this step.
        __syncthreads();
        if (threadIdx.x == 0) st_release(ctl.flags + (size_t)b * kFlagStride, c0 + j + 1);
        if (BWD && s > 1) prefetch_gs(s - 1);   // GS slots of this thread were read above
#pragma unroll
        for (int r = 0; r < PBY; ++r) {
            if (!BWD && !is_boundary(r)) *(VT*)(dst + own0 + (size_t)r * W) = out[r];
            xf[r] = xpass(out[r]);
        }
    }
    if (BWD) {   // the A block ends at s = 1
        if (gs_dead) {   // one more bounded wait for a copy still in flight
            for (long long spins = 0; spins <= kGsSpinLimit && !bar_test(&gs_bar, gs_phase); ++spins) {
            }
        }
        float* q = (float*)R.q + (size_t)species * V;
#pragma unroll
        for (int r = 0; r < PBY; ++r) *(VT*)(q + own0 + (size_t)r * W) = q_out(qacc[r]);
    } else {
        const double t = block_sum((double)qsum, sh);
        if (threadIdx.x == 0) slot(R, P_Q)[b] = t;
        if (b == 0)
            for (int i = threadIdx.x + gridDim.x; i < R.ntiles; i += PTHREADS) slot(R, P_Q)[i] = 0.0;
    }
}

// Host side ---------------------------------------------------------------------------------

bool pers_supported(const Rep& R, int bz, int nw, int nsm) {
    if (R.nx != 128 || R.ny % PBY || R.nz % bz) return false;
    if (!((bz == 16 && nw == 16) || (bz == 8 && nw == 8))) return false;   // one warp per plane
    const int nb = (R.ny / PBY) * (R.nz / bz);
    return nb >= 1 && nb <= nsm * (nw == 8 ? 2 : 1);   // all bricks co-resident
}

int pers_bricks(const Rep& R, int bz) { return (R.ny / PBY) * (R.nz / bz); }

namespace {
template <int BZ, int NW>
cudaError_t pers_attr() {
    const int sm = (int)pers_smem_bytes(4, BZ);
    cudaError_t e = cudaFuncSetAttribute(k_prop_pers<BZ, false, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prop_pers<BZ, true, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_prop_pers<BZ, false, NW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_prop_pers<BZ, true, NW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}
}  // namespace

int pers_prepare(int bz, int nw) {
    if (bz == 16 && nw == 16) return (int)pers_attr<16, 16>();
    if (bz == 8 && nw == 8) return (int)pers_attr<8, 8>();
    return (int)cudaErrorInvalidValue;
}

namespace {
// The SM that runs each CTA of a launch shaped like the sweep (same block size, shared memory
// and cooperative attribute), for the placement of bricks on SMs.
template <int NW>
__global__ void __launch_bounds__(32 * NW, 16 / NW) k_pers_place(int* smid) {
    if (threadIdx.x == 0) {
        unsigned id;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
        smid[blockIdx.x] = (int)id;
    }
}
}  // namespace

int pers_placement(int bz, int nw, int nbricks, int* d_smid, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nbricks);
    cfg.blockDim = dim3(32 * nw);
    cfg.dynamicSmemBytes = pers_smem_bytes(4, bz);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (nw == 16) {
        e = cudaFuncSetAttribute(k_pers_place<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.dynamicSmemBytes);
        if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, k_pers_place<16>, d_smid);
    } else {
        e = cudaFuncSetAttribute(k_pers_place<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.dynamicSmemBytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pers_place<8>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, k_pers_place<8>, d_smid);
    }
    return (int)e;
}

int launch_prop_pers(const Launch& L, bool bwd, int bz, int nw, int nbricks, int* flags, int* abortf, int limit,
                     const int* perm) {
    PersCtl ctl;
    ctl.flags = flags;
    ctl.abort = abortf;
    ctl.status = L.status;
    ctl.perm = perm;
    ctl.limit = limit;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nbricks);
    cfg.blockDim = dim3(32 * nw);
    cfg.dynamicSmemBytes = pers_smem_bytes(4, bz);
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (bz == 16 && nw == 16)
        e = bwd ? cudaLaunchKernelEx(&cfg, k_prop_pers<16, true, 16>, L.reps, ctl)
                : cudaLaunchKernelEx(&cfg, k_prop_pers<16, false, 16>, L.reps, ctl);
    else if (bz == 8 && nw == 8)
        e = bwd ? cudaLaunchKernelEx(&cfg, k_prop_pers<8, true, 8>, L.reps, ctl)
                : cudaLaunchKernelEx(&cfg, k_prop_pers<8, false, 8>, L.reps, ctl);
    else
        e = cudaErrorInvalidValue;
    return (int)e;
}

}  // namespace dscf
