// Persistent contour sweeps (Eq. 16-17) in the whole-row layout (FP32), for one replica or a
// batch of replicas.
//
// One launch runs a whole forward (or backward) sweep of N contour steps.  The lattice is cut
// into bricks of nx x 8 x BZ sites, one brick per CTA (one CTA per SM for BZ = 16, two for
// BZ = 8; the launch is cooperative, so all CTAs are resident together), one warp per plane of
// the brick.  Rows of 96 or 128 sites are held by a whole warp (3 or 4 sites per lane), rows of
// 32, 48 or 64 sites by half a warp (2, 3 or 4 sites per lane), two rows side by side; bricks of
// these narrow rows have 16 rows instead of 8 where ny allows it.  A CTA takes its brick from a
// table (replica, brick, flag base), so replicas of one row width share a launch; a brick waits
// only on the bricks of its own replica.  A warp keeps its plane's x-filtered rows in registers
// from one contour step to the next; per step the CTA only reads the halo rows and planes of its
// eight y/z neighbours from L2, after checking with an acquire load that they have published that
// step.  Per step:
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
// read-modify-written per step.  Each 1-D pass of the separable stencil is one add and one fma
// per site, as packed f32x2 pairs (a scalar tail for three sites per lane), with the centre weight
// folded into the Boltzmann factors.  Every wait is bounded: on timeout the CTA sets a status bit
// and a global abort flag that makes every other CTA stop waiting, so the launch always finishes.
#include "dscf_internal.cuh"

#include <algorithm>

namespace dscf {

namespace {

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

struct PersCtl {
    int* flags;          // one step counter per brick, kFlagStride ints apart
    int* abort;          // set by a CTA that gave up waiting
    int* status;         // device status word
    const int4* table;   // per CTA: replica, brick in the replica, flag index of the replica's brick 0
    int limit;           // polls before giving up
};

// Wait until every neighbour brick has published `target`; threads 0..7 poll one neighbour each
// (each counter on its own cache line).  Only the pollers look at the shared abort flag, and only
// every 32 polls, so that the waits of all CTAs do not contend on one line.
__device__ __forceinline__ void wait_nb(const PersCtl& c, const int* nb, unsigned target, bool& aborted) {
    if (threadIdx.x < 8 && !aborted) {
        const int* f = c.flags + (size_t)nb[threadIdx.x] * kFlagStride;
        int spins = 0;
        while ((int)((unsigned)ld_acquire(f) - target) < 0) {   // wrap-safe: counters only grow
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

template <int BZ, int PBY>
struct PersGeom {
    static constexpr int NH = 2 * (BZ + 2) + 2 * PBY;   // halo rows per step
};

// Row geometry of a brick of width W and PBY rows: a row is held by LPR lanes, VEC consecutive
// sites each; a warp holds HALVES rows side by side (lanes 0..LPR-1 the first, LPR..31 the
// second), so each lane carries RPL of the plane's PBY rows (rows h RPL .. h RPL + RPL - 1 for
// lane half h).
template <int W, int PBY>
struct PRow {
    static constexpr int LPR = (W == 96 || W == 128) ? 32 : 16;
    static constexpr int VEC = W / LPR;
    static constexpr int HALVES = 32 / LPR;
    static constexpr int RPL = PBY / HALVES;
    static constexpr int CH = W / 4;   // 16-byte chunks per row
    static_assert(LPR * VEC == W && VEC >= 2 && VEC <= 4, "row width");
    static_assert(HALVES * CH <= 32, "one 16-byte chunk per lane for the rows a warp copies");
};

// VEC consecutive FP32 values: one vector access for 2 and 4, three scalar ones for 3
template <int VEC>
__device__ __forceinline__ void ldv(const float* p, float (&v)[VEC]) {
    if constexpr (VEC == 4) {
        const float4 t = *(const float4*)p;
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if constexpr (VEC == 2) {
        const float2 t = *(const float2*)p;
        v[0] = t.x; v[1] = t.y;
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) v[k] = p[k];
    }
}
template <int VEC>
__device__ __forceinline__ void stv(float* p, const float (&v)[VEC]) {
    if constexpr (VEC == 4) {
        *(float4*)p = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (VEC == 2) {
        *(float2*)p = make_float2(v[0], v[1]);
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) p[k] = v[k];
    }
}
// o = c + r (a + d) per site: packed pairs, a scalar tail for odd VEC (same rounding: one add, one
// fma per site either way)
template <int VEC>
__device__ __forceinline__ void mixv(const float (&a)[VEC], const float (&c)[VEC], const float (&d)[VEC], float rr,
                                     unsigned long long rr2, float (&o)[VEC]) {
#pragma unroll
    for (int k = 0; k + 1 < VEC; k += 2)
        upk2(fma2(rr2, add2(pk2(a[k], a[k + 1]), pk2(d[k], d[k + 1])), pk2(c[k], c[k + 1])), o[k], o[k + 1]);
    if constexpr (VEC & 1) o[VEC - 1] = __fmaf_rn(rr, __fadd_rn(a[VEC - 1], d[VEC - 1]), c[VEC - 1]);
}
// o = s * v per site
template <int VEC>
__device__ __forceinline__ void mulv(const float (&s)[VEC], const float (&v)[VEC], float (&o)[VEC]) {
#pragma unroll
    for (int k = 0; k + 1 < VEC; k += 2) upk2(mul2(pk2(s[k], s[k + 1]), pk2(v[k], v[k + 1])), o[k], o[k + 1]);
    if constexpr (VEC & 1) o[VEC - 1] = __fmul_rn(s[VEC - 1], v[VEC - 1]);
}
// q += g * v per site
template <int VEC>
__device__ __forceinline__ void fmav(const float (&g)[VEC], const float (&v)[VEC], float (&q)[VEC]) {
#pragma unroll
    for (int k = 0; k + 1 < VEC; k += 2)
        upk2(fma2(pk2(g[k], g[k + 1]), pk2(v[k], v[k + 1]), pk2(q[k], q[k + 1])), q[k], q[k + 1]);
    if constexpr (VEC & 1) q[VEC - 1] = __fmaf_rn(g[VEC - 1], v[VEC - 1], q[VEC - 1]);
}
// scalar c times each site
template <int VEC>
__device__ __forceinline__ void scalev(float c, unsigned long long c2, float (&v)[VEC]) {
#pragma unroll
    for (int k = 0; k + 1 < VEC; k += 2) upk2(mul2(c2, pk2(v[k], v[k + 1])), v[k], v[k + 1]);
    if constexpr (VEC & 1) v[VEC - 1] = __fmul_rn(c, v[VEC - 1]);
}

}  // namespace

size_t pers_smem_bytes(int width, int pby, int bz) {
    const size_t PBY = (size_t)pby;
    // YS (y-filtered level, planes -1..bz) + XH (x-filtered y-halo rows of the own planes) + ZH
    // (x-filtered z-halo planes, rows -1..pby) + halo staging + backward G_s of the brick
    const size_t rows = (size_t)(bz + 2) * PBY + 2 * (size_t)bz + 2 * (PBY + 2) + (2 * (bz + 2) + 2 * PBY) +
                        (size_t)bz * PBY;
    return rows * (size_t)width * sizeof(float);
}

// Warp w owns plane w of the brick, all PBY rows (HALVES rows side by side), VEC sites of each
// row per lane; the x-filtered rows of the previous level stay in its registers, so the y pass
// runs in registers (the rows across the lane halves by one shuffle, the two y-halo rows of the
// plane from shared memory) and only the y-filtered rows go through shared memory, for the z pass
// of the neighbouring planes.  The z-halo planes are y-filtered one row per lane half.  Brick-
// boundary values are stored and published first; the rest of the forward G_s follows without a
// fence (the backward G+ interior is never stored: it stays in registers).
// Each CTA takes its brick from the table, so several replicas run in one launch (of one row
// width here; the mixed-width kernel below calls this per CTA), each brick waiting only on the
// bricks of its own replica.
template <int W, int PBY, int BZ, bool BWD, int NW>
__device__ __forceinline__ void pers_sweep(const Rep* __restrict__ reps, const PersCtl& ctl) {
    static_assert(NW == BZ, "one warp per plane");
    using RG = PRow<W, PBY>;
    constexpr int VEC = RG::VEC, LPR = RG::LPR, HALVES = RG::HALVES, RPL = RG::RPL, CH = RG::CH;
    constexpr int PWARPS = NW;
    using G = PersGeom<BZ, PBY>;
    extern __shared__ __align__(16) unsigned char smem[];
    float* YS = (float*)smem;                                  // [BZ+2][PBY][W]
    float* XH = YS + (BZ + 2) * PBY * W;                       // [2][BZ][W]   rows -1 and PBY
    float* ZH = XH + 2 * BZ * W;                               // [2][PBY+2][W] planes -1 and BZ
    float* HS = ZH + 2 * (PBY + 2) * W;                        // [NH][W]
    float* GS = HS + G::NH * W;                                // [BZ][PBY][W] backward G_s
    __shared__ double sh[33];
    __shared__ int nbs[8];
    __shared__ __align__(8) unsigned long long gs_bar;   // backward: completion of the G_s prefetch
    const int4 tb = ctl.table[blockIdx.x];
    const Rep& R = reps[tb.x];
    const int b = tb.y;
    const int fown = tb.z + tb.y;   // own step counter
    const int ny = R.ny, nz = R.nz, N = R.N, nA = R.nA;
    const int plane = W * ny;
    const size_t V = (size_t)R.V;
    const int nby = ny / PBY, nbz = nz / BZ;
    const int by = b % nby, bz = b / nby;
    const int y0 = by * PBY, z0 = bz * BZ;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int hf = lane / LPR, li = lane - hf * LPR;   // lane half (row group) and lane within the row
    const int xo = VEC * li;
    const int seg = lane - li;
    const int lsrc = seg + ((li + LPR - 1) & (LPR - 1)), rsrc = seg + ((li + 1) & (LPR - 1));
    // Each 1-D pass is applied as c + r (a + d) with r = alpha / (1 - 2 alpha), i.e. the
    // stencil's pass divided by its centre weight be = 1 - 2 alpha; the three passes then give
    // sigma / be^3, and be^3 is folded into the Boltzmann factors (and into q at its write-out).
    const double be_d = 1.0 - 2.0 * R.alpha;
    const float rr = (float)(R.alpha / be_d), be3 = (float)(be_d * be_d * be_d);
    const unsigned long long rr2 = pk2(rr, rr), be32 = pk2(be3, be3);
    if (threadIdx.x < 8) {
        const int k = threadIdx.x < 4 ? threadIdx.x : threadIdx.x + 1;   // skip the centre
        const int dy = k % 3 - 1, dz = k / 3 - 1;
        nbs[threadIdx.x] = tb.z + (by + dy + nby) % nby + nby * ((bz + dz + nbz) % nbz);
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
    for (int h = threadIdx.x; h < G::NH; h += 32 * PWARPS) {
        int r, pl;
        halo_rp(h, r, pl);
        const int y = (y0 + r + ny) % ny, z = (z0 + pl + nz) % nz;
        hoff[h] = z * plane + y * W;
    }
    // step counters of a replica's bricks are equal at launch (unsigned: they may wrap in long runs)
    const unsigned c0 = (unsigned)ctl.flags[(size_t)fown * kFlagStride];
    bool aborted = ld_acquire(ctl.abort) != 0;

    auto xpass = [&](const float (&v)[VEC], float (&o)[VEC]) {   // x pass of a periodic row: v + r (left + right)
        const float lv = __shfl_sync(0xffffffffu, v[VEC - 1], lsrc);
        const float rv = __shfl_sync(0xffffffffu, v[0], rsrc);
        float a[VEC], d[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            a[k] = k ? v[k - 1] : lv;
            d[k] = (k + 1 < VEC) ? v[k + 1] : rv;
        }
        mixv<VEC>(a, v, d, rr, rr2, o);
    };
    auto ys = [&](int pl, int r) { return YS + ((pl + 1) * PBY + r) * W + xo; };
    const bool face_plane = (w == 0 || w == BZ - 1);
    auto is_boundary = [&](int r) { return face_plane || r == 0 || r == PBY - 1; };
    // own plane never wraps: offset of (row r, plane w) is own0 + r * W
    const size_t own0 = (size_t)(z0 + w) * plane + (size_t)y0 * W + xo;
    auto row_of = [&](int p) { return hf * RPL + p; };

    float e[RPL][VEC];
    auto load_e = [&](int species) {
        const float* E = (const float*)R.E + (size_t)species * V;
#pragma unroll
        for (int p = 0; p < RPL; ++p) {
            ldv<VEC>(E + own0 + (size_t)row_of(p) * W, e[p]);
            scalev<VEC>(be3, be32, e[p]);
        }
    };
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
    float xf[RPL][VEC];
#pragma unroll
    for (int p = 0; p < RPL; ++p)
#pragma unroll
        for (int k = 0; k < VEC; ++k) xf[p][k] = one;
    for (int i = threadIdx.x; i < (2 * BZ + 2 * (PBY + 2)) * W; i += 32 * PWARPS) XH[i] = one;   // XH and ZH
    float qacc[BWD ? RPL : 1][VEC];
#pragma unroll
    for (int p = 0; p < (BWD ? RPL : 1); ++p)
#pragma unroll
        for (int k = 0; k < VEC; ++k) qacc[p][k] = 0.f;
    float qsum = 0.f;
    int species = BWD ? (N <= nA ? 0 : 1) : (1 <= nA ? 0 : 1);
    load_e(species);
    if (BWD) {
        if (threadIdx.x == 0) bar_init(&gs_bar);
        __syncthreads();
        prefetch_gs(N);
    }
    __syncthreads();

    auto write_q = [&](int sp) {   // a block's quadrature, scaled back by be^3
        float* q = (float*)R.q + (size_t)sp * V;
#pragma unroll
        for (int p = 0; p < (BWD ? RPL : 1); ++p) {
            float o[VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) o[k] = qacc[p][k];
            scalev<VEC>(be3, be32, o);
            stv<VEC>(q + own0 + (size_t)row_of(p) * W, o);
#pragma unroll
            for (int k = 0; k < VEC; ++k) qacc[p][k] = 0.f;
        }
    };

    for (int j = 0; j < N; ++j) {
        const int s = BWD ? N - j : j + 1;
        const int sp = (s <= nA) ? 0 : 1;
        if (sp != species) {
            if (BWD) write_q(species);   // leaving the B block: its quadrature is complete
            species = sp;
            load_e(species);
        }
        // halo of the previous step, x-filtered into XH / ZH; each warp copies and filters the
        // rows of its own lane halves (a __syncwarp makes every lane's copied chunk visible)
        if (j > 0) {
            wait_nb(ctl, nbs, c0 + (unsigned)j, aborted);
            const float* src = BWD ? (const float*)(((j - 1) & 1) ? R.Gp1 : R.Gp0)
                                   : (const float*)R.G + (size_t)(s - 2) * V;
            {
                const int i = lane / CH, ch = lane - i * CH;
                for (int h0 = w * HALVES; h0 < G::NH; h0 += PWARPS * HALVES)
                    if (i < HALVES) cp16(HS + (h0 + i) * W + 4 * ch, src + hoff[h0 + i] + 4 * ch);
            }
            cpc();
            cpw0();
            __syncwarp();
            for (int h0 = w * HALVES; h0 < G::NH; h0 += PWARPS * HALVES) {
                const int h = h0 + hf;
                float v[VEC], o[VEC];
                ldv<VEC>(HS + h * W + xo, v);
                xpass(v, o);
                int r, pl;
                halo_rp(h, r, pl);
                stv<VEC>(halo_dst(r, pl) + xo, o);
            }
        }
        __syncthreads();
        // y pass of the own plane in registers (its two y-halo rows from XH), into YS
        {
            float up[VEC], dn[VEC];   // the row above the lane's first row, below its last
            ldv<VEC>(XH + w * W + xo, up);           // row -1
            ldv<VEC>(XH + (BZ + w) * W + xo, dn);    // row PBY
            if constexpr (HALVES == 2) {   // rows across the two lane halves
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    const float last = __shfl_xor_sync(0xffffffffu, xf[RPL - 1][k], LPR);
                    const float first = __shfl_xor_sync(0xffffffffu, xf[0][k], LPR);
                    if (hf == 1) up[k] = last;
                    else dn[k] = first;
                }
            }
            float prev[VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) prev[k] = up[k];
#pragma unroll
            for (int p = 0; p < RPL; ++p) {
                float yv[VEC], cur[VEC];
#pragma unroll
                for (int k = 0; k < VEC; ++k) cur[k] = xf[p][k];
                if (p + 1 < RPL) mixv<VEC>(prev, cur, xf[p + 1 < RPL ? p + 1 : p], rr, rr2, yv);
                else mixv<VEC>(prev, cur, dn, rr, rr2, yv);
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    prev[k] = cur[k];
                    xf[p][k] = yv[k];   // xf now holds the y-filtered rows
                }
                stv<VEC>(ys(w, row_of(p)), yv);
            }
        }
        // y pass of the z-halo planes, one row per lane half (PBY rows of each of the two planes)
        for (int t0 = w * HALVES; t0 < 2 * PBY; t0 += PWARPS * HALVES) {
            const int t = t0 + hf;
            const int side = t / PBY, r = t % PBY;
            const float* zr = ZH + (side * (PBY + 2) + r + 1) * W + xo;
            float a[VEC], c[VEC], d[VEC], o[VEC];
            ldv<VEC>(zr - W, a);
            ldv<VEC>(zr, c);
            ldv<VEC>(zr + W, d);
            mixv<VEC>(a, c, d, rr, rr2, o);
            stv<VEC>(ys(side ? BZ : -1, r), o);
        }
        __syncthreads();
        // z pass and step output
        float* dst = BWD ? (float*)((j & 1) ? R.Gp1 : R.Gp0) : (float*)R.G + (size_t)(s - 1) * V;
        if (BWD) wait_gs();
        float out[RPL][VEC];
#pragma unroll
        for (int p = 0; p < RPL; ++p) {
            const int r = row_of(p);
            float a[VEC], d[VEC], sg[VEC];
            ldv<VEC>(ys(w - 1, r), a);
            ldv<VEC>(ys(w + 1, r), d);
            mixv<VEC>(a, xf[p], d, rr, rr2, sg);
            mulv<VEC>(e[p], sg, out[p]);
            if constexpr (BWD) {
                float g[VEC];
                ldv<VEC>(GS + (w * PBY + r) * W + xo, g);
                fmav<VEC>(g, sg, qacc[p]);
            } else {
                if (s == N) {
                    float t = out[p][0] + out[p][1];
                    if constexpr (VEC == 3) t = t + out[p][2];
                    if constexpr (VEC == 4) t = t + (out[p][2] + out[p][3]);
                    qsum += t;
                }
            }
            if (is_boundary(r) && (!BWD || s > 1)) stv<VEC>(dst + own0 + (size_t)r * W, out[p]);
        }
        // publish the boundary of this step: the CTA barrier orders every thread's boundary stores
        // before thread 0's release store, and release is cumulative, so a CTA whose acquire load
        // reads the new counter sees them.  The barrier also ends every warp's reads of YS, XH
        // and ZH for this step.
        __syncthreads();
        if (threadIdx.x == 0) st_release(ctl.flags + (size_t)fown * kFlagStride, (int)(c0 + (unsigned)j + 1u));
        if (BWD && s > 1) prefetch_gs(s - 1);   // GS slots of this thread were read above
#pragma unroll
        for (int p = 0; p < RPL; ++p) {
            if (!BWD && !is_boundary(row_of(p))) stv<VEC>(dst + own0 + (size_t)row_of(p) * W, out[p]);
            xpass(out[p], xf[p]);
        }
    }
    if (BWD) {   // the A block ends at s = 1
        if (gs_dead) {   // one more bounded wait for a copy still in flight
            for (long long spins = 0; spins <= kGsSpinLimit && !bar_test(&gs_bar, gs_phase); ++spins) {
            }
        }
        write_q(species);
    } else {
        const double t = block_sum((double)qsum, sh);
        const int bl = ctl.table[blockIdx.x].y;   // reloaded: not kept live through the sweep
        if (threadIdx.x == 0) slot(R, P_Q)[bl] = t;
        if (bl == 0) {   // slots past the replica's bricks (the propagator tiling may have more)
            const int nb = nby * nbz;
            for (int i = threadIdx.x + nb; i < R.ntiles; i += 32 * PWARPS) slot(R, P_Q)[i] = 0.0;
        }
    }
}


template <int W, int PBY, int BZ, bool BWD, int NW>
__global__ void __launch_bounds__(32 * NW, 16 / NW) k_prop_pers(const Rep* __restrict__ reps, PersCtl ctl) {
    pers_sweep<W, PBY, BZ, BWD, NW>(reps, ctl);
}

// Bricks of several row widths (32 to 96 sites) in one launch (batches): each CTA runs the sweep of
// its replica's width; the launch's dynamic shared memory covers the largest.  128-wide replicas
// keep launches of their own (with them in the same function the registers would spill).
template <int BZ, bool BWD, int NW>
__global__ void __launch_bounds__(32 * NW, 16 / NW) k_prop_pers_mix(const Rep* __restrict__ reps, PersCtl ctl) {
    const Rep& R = reps[ctl.table[blockIdx.x].x];
    const int pby = pers_pby_of(R.nx, R.ny);
    switch (R.nx * 32 + pby) {
        case 32 * 32 + 8: pers_sweep<32, 8, BZ, BWD, NW>(reps, ctl); break;
        case 32 * 32 + 16: pers_sweep<32, 16, BZ, BWD, NW>(reps, ctl); break;
        case 48 * 32 + 8: pers_sweep<48, 8, BZ, BWD, NW>(reps, ctl); break;
        case 48 * 32 + 16: pers_sweep<48, 16, BZ, BWD, NW>(reps, ctl); break;
        case 64 * 32 + 8: pers_sweep<64, 8, BZ, BWD, NW>(reps, ctl); break;
        case 64 * 32 + 16: pers_sweep<64, 16, BZ, BWD, NW>(reps, ctl); break;
        case 96 * 32 + 8: pers_sweep<96, 8, BZ, BWD, NW>(reps, ctl); break;
        default: break;   // not reached: the host builds mixed launches of these widths only
    }
}

// Host side ---------------------------------------------------------------------------------

bool pers_width_ok(int nx) { return nx == 32 || nx == 48 || nx == 64 || nx == 96 || nx == 128; }

int pers_pby(const Rep& R) { return pers_pby_of(R.nx, R.ny); }

size_t pers_mix_smem_bytes(int bz) {
    size_t m = 0;
    for (int w : {32, 48, 64}) m = std::max(m, pers_smem_bytes(w, 16, bz));
    for (int w : {32, 48, 64, 96}) m = std::max(m, pers_smem_bytes(w, 8, bz));
    return m;
}

// Brick depths: 16 planes on 16 warps (one CTA per SM) or 8 planes on 8 warps (two CTAs per SM).
bool pers_supported(const Rep& R, int bz, int nw, int nsm) {
    if (!pers_width_ok(R.nx) || R.ny % 8 || R.nz % bz) return false;
    if (!((bz == 16 && nw == 16) || (bz == 8 && nw == 8))) return false;   // one warp per plane
    const int nb = pers_bricks(R, bz);
    return nb >= 1 && nb <= nsm * (nw == 8 ? 2 : 1);   // all bricks co-resident
}

int pers_bricks(const Rep& R, int bz) { return (R.ny / pers_pby(R)) * (R.nz / bz); }

namespace {
template <int W, int PBY, int BZ, int NW>
cudaError_t pers_attr() {
    const int sm = (int)pers_smem_bytes(W, PBY, BZ);
    cudaError_t e = cudaFuncSetAttribute(k_prop_pers<W, PBY, BZ, false, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_prop_pers<W, PBY, BZ, true, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_prop_pers<W, PBY, BZ, false, NW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_prop_pers<W, PBY, BZ, true, NW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}
template <int BZ, int NW>
cudaError_t pers_mix_attr() {
    const int sm = (int)pers_mix_smem_bytes(BZ);
    cudaError_t e = cudaFuncSetAttribute(k_prop_pers_mix<BZ, false, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_prop_pers_mix<BZ, true, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_prop_pers_mix<BZ, false, NW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_prop_pers_mix<BZ, true, NW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}
}  // namespace

// ACTION(W, PBY, BZ, NW) for the instantiated (width, rows) pairs of one brick depth
#define DSCF_PERS_SWITCH(BB, NN, ACTION)                          \
    switch (width * 32 + pby) {                                  \
        case 128 * 32 + 8: ACTION(128, 8, BB, NN); break;        \
        case 96 * 32 + 8: ACTION(96, 8, BB, NN); break;          \
        case 64 * 32 + 8: ACTION(64, 8, BB, NN); break;          \
        case 64 * 32 + 16: ACTION(64, 16, BB, NN); break;        \
        case 48 * 32 + 8: ACTION(48, 8, BB, NN); break;          \
        case 48 * 32 + 16: ACTION(48, 16, BB, NN); break;        \
        case 32 * 32 + 8: ACTION(32, 8, BB, NN); break;          \
        case 32 * 32 + 16: ACTION(32, 16, BB, NN); break;        \
        default: break;                                          \
    }

int pers_prepare(int width, int pby, int bz, int nw) {
    cudaError_t e = cudaErrorInvalidValue;
#define DSCF_PERS_ATTR(WW, PP, BB, NN) e = pers_attr<WW, PP, BB, NN>()
    if (bz == 16 && nw == 16) {
        if (width == 0) e = pers_mix_attr<16, 16>();
        else DSCF_PERS_SWITCH(16, 16, DSCF_PERS_ATTR)
    } else if (bz == 8 && nw == 8) {
        if (width == 0) e = pers_mix_attr<8, 8>();
        else DSCF_PERS_SWITCH(8, 8, DSCF_PERS_ATTR)
    }
#undef DSCF_PERS_ATTR
    return (int)e;
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
    cfg.dynamicSmemBytes = pers_smem_bytes(128, 8, bz);
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

int launch_prop_pers(const Launch& L, bool bwd, int width, int pby, int bz, int nw, int nbricks, const int4* table,
                     int* flags, int* abortf, int limit) {
    PersCtl ctl;
    ctl.flags = flags;
    ctl.abort = abortf;
    ctl.status = L.status;
    ctl.table = table;
    ctl.limit = limit;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nbricks);
    cfg.blockDim = dim3(32 * nw);
    cfg.dynamicSmemBytes = width ? pers_smem_bytes(width, pby, bz) : pers_mix_smem_bytes(bz);
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaErrorInvalidValue;
#define DSCF_PERS_LAUNCH(WW, PP, BB, NN)                                                                  \
    e = bwd ? cudaLaunchKernelEx(&cfg, k_prop_pers<WW, PP, BB, true, NN>, L.reps, ctl)                    \
            : cudaLaunchKernelEx(&cfg, k_prop_pers<WW, PP, BB, false, NN>, L.reps, ctl)
    if (bz == 16 && nw == 16) {
        if (width == 0)
            e = bwd ? cudaLaunchKernelEx(&cfg, k_prop_pers_mix<16, true, 16>, L.reps, ctl)
                    : cudaLaunchKernelEx(&cfg, k_prop_pers_mix<16, false, 16>, L.reps, ctl);
        else DSCF_PERS_SWITCH(16, 16, DSCF_PERS_LAUNCH)
    } else if (bz == 8 && nw == 8) {
        if (width == 0)
            e = bwd ? cudaLaunchKernelEx(&cfg, k_prop_pers_mix<8, true, 8>, L.reps, ctl)
                    : cudaLaunchKernelEx(&cfg, k_prop_pers_mix<8, false, 8>, L.reps, ctl);
        else DSCF_PERS_SWITCH(8, 8, DSCF_PERS_LAUNCH)
    }
#undef DSCF_PERS_LAUNCH
    return (int)e;
}
#undef DSCF_PERS_SWITCH

}  // namespace dscf
