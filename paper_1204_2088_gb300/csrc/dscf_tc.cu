// Forward 5^3 circular convolution of the learned predictor on the 5th-generation tensor cores
// (tcgen05: operands in shared memory, FP32 accumulators in tensor memory), for grids whose x
// extent is a multiple of 128.
//
// GEMM view: for an output row of 128 sites along x, D[x][co] = sum over the 125 offsets
// (dz, dy, dx) and input channels ci of A[x][ci] B[co][ci] with A the input row (y+dy, z+dz)
// shifted by dx.  A CTA computes R output rows (y0..y0+R-1, z, x0..x0+127) into TMEM accumulators
// of 128 lanes x CO columns.  For each dz the R + 4 input rows y0-2..y0+R+1 of plane z+dz
// (periodic) sit in shared memory in the no-swizzle K-major operand layout
//   [row][channel group of 8][x' = 0..131][8 channels]  (x' = x - x0 + 2),
// in which 8 consecutive sites of one channel group form a contiguous 128-byte core matrix: the
// descriptor has 128 B between core matrices along M (sites) and 132 x 16 B between channel
// groups along K, and the shift by dx is just 16 dx bytes added to its start address.  Weights
// are staged as [offset][channel group][co][8], the same layout for the N x K operand.  One
// thread issues the MMAs; tcgen05.commit on mbarriers tells the copying warp when staged operands
// may be overwritten and the CTA when the accumulators are complete.  The epilogue (bias, then
// tanh to BF16 or FP32 stores) reads each warp's quarter of the TMEM lanes with tcgen05.ld.
//
// The first layer (2 input channels, R = 4) folds the five x offsets into 16 channels and is a
// persistent, warp-specialised kernel: bulk (TMA) copies, MMAs and epilogue of successive tiles
// overlap.  The 32-channel layers stack the five dy offsets along N (R = 8) and stream each
// plane's rows in, one bulk copy per row and channel group.  Activations between layers are
// stored in a padded channel-group layout (each row's channel groups contiguous, with periodic
// copies of two sites at each end) so that every staged row is one contiguous run.
//
// Every wait is bounded; a CTA that gives up sets the error word, frees its tensor memory and
// returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "dscf_internal.cuh"

namespace dscf {

namespace {

typedef __nv_bfloat16 bf16;

constexpr int TC_R = 4;            // output rows per tile of the first layer
constexpr int TC_XP = 132;         // staged row length (128 + 2 on each side)
constexpr long long kTcSpinLimit = 1ll << 20;   // try_wait polls (each may suspend ~1 us)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (no swizzle): start address, leading-dimension byte offset
// (between core matrices along K), stride-dimension byte offset (between 8-row core-matrix
// groups along M or N), descriptor version 1 in bits 46-47.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B (bits 7-9
// and 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* mbar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ int mbar_try_wait(uint64_t* mbar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred P1;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return (int)done;
}
// Bounded wait on an mbarrier phase; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
    for (long long i = 0; i < kTcSpinLimit; ++i)
        if (mbar_try_wait(mbar, parity)) return true;
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(mbar)) : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ int wrapi_(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// Bulk (TMA) copies global -> shared completing on an mbarrier: both addresses 16-byte aligned,
// bytes a multiple of 16.
__device__ __forceinline__ void mbar_expect(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}

// Store the 32 BF16 channels hv of site x of grid row rowi ((b nz + z) ny + y) in the padded
// channel-group layout [rows][4][nx + 4][8] that the next layer stages from: site x at x + 2, and
// the two sites at each end of the row also as the periodic copies beyond the other end.
__device__ __forceinline__ void store_padded32(bf16* __restrict__ out, size_t rowi, int x, int nx, const bf16* hv) {
    bf16* base = out + rowi * 4 * (size_t)(nx + 4) * 8;
    const int xh = x < 2 ? x + nx + 2 : (x >= nx - 2 ? x - nx + 2 : -1);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        bf16* row = base + (size_t)g * (nx + 4) * 8;
        *(uint4*)(row + (size_t)(x + 2) * 8) = ((const uint4*)hv)[g];
        if (xh >= 0) *(uint4*)(row + (size_t)xh * 8) = ((const uint4*)hv)[g];
    }
}

// First layer (2 -> 32 channels, tanh) on the folded input: channels 2 dx + ci (dx = 0..4,
// ci = 0..1) hold the two real input channels at x + dx - 2 (zero in channels 10..15), so one
// K = 16 step covers all five x offsets and the offsets left are the 25 (dz, dy).  The folded
// input is stored by channel group within each x row, with two periodic copies on each side,
// in: [B][nz][ny][2][nx + 4][8] BF16 (site x at x + 2), so that each group's part of a staged row
// (the tile's 128 sites and two on each side) is one contiguous 2112-byte run: one bulk copy.
// wt: [dz][dy][k / 8][co][k % 8] BF16, staged once per CTA.
// Persistent: each CTA takes tiles (4 output rows of 128 sites) blockIdx.x, + gridDim.x, ... and
// streams their planes (5 per tile) through two staging buffers, with warp-specialised roles
// synchronised by mbarriers only:
//   warp 1 (copies)   fills a buffer (16 bulk copies, `full`) as soon as the MMAs that read it
//                     have completed (`freed`), so the next plane is in flight while one is used;
//   thread 0 (MMAs)   issues the 20 MMAs (M = 128, N = 32, K = 16) of each plane into one of two
//                     accumulator sets in TMEM (alternating by tile) and commits `tfull` after a
//                     tile's last plane, once the epilogue has released that set (`tfree`);
//   warps 2..5        (one TMEM lane quarter each) read a finished set, apply tanh(acc + bias),
//                     store BF16 in the padded channel-group layout of the next layer's input
//                     ([B][nz][ny][4][nx + 4][8]) and release the set,
// so the copies, the MMAs and the epilogue of successive tiles overlap.
constexpr int L1_G = 2;                            // channel groups of the folded input
constexpr int L1_CO = 32;
constexpr int L1_ROWB = L1_G * TC_XP * 16;         // bytes of one staged row
constexpr int L1_ABYTES = (TC_R + 4) * L1_ROWB;    // one plane's staged rows
constexpr int L1_WBYTES = 25 * L1_G * L1_CO * 16;  // weights of the 25 (dz, dy)
constexpr int L1_THREADS = 192;                    // warps: MMA issue, copies, 4 epilogue
constexpr int L1_TMEM_COLS = 256;                  // two accumulator sets of TC_R x 32 columns
constexpr int L1_CTAS_PER_SM = 2;

__global__ void __launch_bounds__(L1_THREADS, L1_CTAS_PER_SM)
    k_conv_tc_l1(const bf16* __restrict__ in, const bf16* __restrict__ wt, const float* __restrict__ bias, int cout,
                 bf16* __restrict__ out, int nx, int ny, int nz, int B, int* __restrict__ err) {
    constexpr int CO = L1_CO;
    constexpr uint32_t IDESC = idesc_bf16(128, CO);
    static_assert(2 * TC_R * CO <= L1_TMEM_COLS, "accumulators exceed the tensor-memory allocation");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* Ws = smem + 2 * L1_ABYTES;
    __shared__ __align__(8) uint64_t full[2], freed[2], tfull[2], tfree[2], wbar;
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nxt = nx / 128, nyb = ny / TC_R;
    const int ntile = B * nz * nyb * nxt;
    const int nk = ntile > (int)blockIdx.x ? (ntile - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    const size_t V = (size_t)nx * ny * nz;
    // tile t -> sample b, plane z, first row y0, first site x0
    auto tile_of = [&](int k, int& b, int& z, int& y0, int& x0) {
        int t = (int)blockIdx.x + k * (int)gridDim.x;
        x0 = (t % nxt) * 128;
        t /= nxt;
        y0 = (t % nyb) * TC_R;
        t /= nyb;
        z = t % nz;
        b = t / nz;
    };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(L1_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&freed[i], 1);
            mbar_init(&tfull[i], 1);
            mbar_init(&tfree[i], 4);   // one arrival per epilogue warp
        }
        mbar_init(&wbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;

    bool ok = true;
    int nfill0 = 0, nfill1 = 0;   // fills issued per buffer
    if (warp == 1) {   // bulk copies: the weights, then the 5 planes of each tile in order
        if (lane == 0) {
            mbar_expect(&wbar, L1_WBYTES);
            bulk_g2s(Ws, wt, L1_WBYTES, &wbar);
        }
        for (int p = 0; p < 5 * nk && ok; ++p) {
            const int buf = p & 1;
            if (p >= 2) {
                ok = __all_sync(0xffffffffu, mbar_wait(&freed[buf], (uint32_t)(((p >> 1) - 1) & 1)));
                if (!ok) break;
            }
            int b, z, y0, x0;
            tile_of(p / 5, b, z, y0, x0);
            const int zin = wrapi_(z + p % 5 - 2, nz);
            const bf16* inb = in + (size_t)b * (V / nx) * 2 * (nx + 4) * 8;
            unsigned char* A = smem + buf * L1_ABYTES;
            if (lane == 0) mbar_expect(&full[buf], L1_ABYTES);
            __syncwarp();
            if (lane < (TC_R + 4) * L1_G) {   // one staged row of one channel group per lane
                const int i = lane / L1_G, g = lane % L1_G;
                const int yin = wrapi_(y0 - 2 + i, ny);
                const bf16* src = inb + ((((size_t)zin * ny + yin) * L1_G + g) * (nx + 4) + x0) * 8;
                bulk_g2s(A + (i * L1_G + g) * TC_XP * 16, src, TC_XP * 16, &full[buf]);
            }
            if (buf) ++nfill1;
            else ++nfill0;
        }
        if (!ok && lane == 0) atomicOr(err, 1);
    } else if (tid == 0) {   // MMA issue
        ok = mbar_wait(&wbar, 0u);
        for (int k = 0; k < nk && ok; ++k) {
            const int acc = k & 1;
            if (k >= 2 && !(ok = mbar_wait(&tfree[acc], (uint32_t)(((k >> 1) - 1) & 1)))) break;
            fence_after_sync();
            const uint32_t t0 = tmem + (uint32_t)(acc * TC_R * CO);
            for (int dzi = 0; dzi < 5; ++dzi) {
                const int p = 5 * k + dzi, buf = p & 1;
                if (!(ok = mbar_wait(&full[buf], (uint32_t)((p >> 1) & 1)))) break;
                fence_after_sync();
                const uint32_t a0 = smem_u32(smem + buf * L1_ABYTES);
                const uint32_t w0 = smem_u32(Ws) + (uint32_t)(dzi * 5 * L1_G * CO * 16);
                for (int r = 0; r < TC_R; ++r)
                    for (int dyi = 0; dyi < 5; ++dyi) {
                        const uint32_t aaddr = a0 + (uint32_t)(((r + dyi) * L1_G) * TC_XP + 2) * 16u;
                        const uint32_t baddr = w0 + (uint32_t)(dyi * L1_G * CO) * 16u;
                        mma_bf16(t0 + (uint32_t)(r * CO), smem_desc(aaddr, TC_XP * 16, 128),
                                 smem_desc(baddr, CO * 16, 128), IDESC, (dzi | dyi) != 0);
                    }
                mma_commit(&freed[buf]);   // the buffer may be refilled
            }
            if (ok) mma_commit(&tfull[acc]);   // the tile's accumulators are complete
        }
        if (!ok) atomicOr(err, 1);
    } else if (warp >= 2) {   // epilogue: warp w reads TMEM lane quarter w % 4
        const int q = warp & 3;
        float bs[CO];
#pragma unroll
        for (int co = 0; co < CO; ++co) bs[co] = co < cout ? bias[co] : 0.f;
        for (int k = 0; k < nk && ok; ++k) {
            const int acc = k & 1;
            ok = __all_sync(0xffffffffu, mbar_wait(&tfull[acc], (uint32_t)((k >> 1) & 1)));
            if (!ok) break;
            fence_after_sync();
            int b, z, y0, x0;
            tile_of(k, b, z, y0, x0);
            const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * TC_R * CO);
#pragma unroll 1
            for (int r = 0; r < TC_R; ++r) {
                float v[CO];
                tmem_ld32(tq + (uint32_t)(r * CO), v);
                __align__(16) bf16 hv[CO];
#pragma unroll
                for (int co = 0; co < CO; ++co) hv[co] = __float2bfloat16(tanhf(v[co] + bs[co]));
                store_padded32(out, ((size_t)b * nz + z) * ny + y0 + r, x0 + q * 32 + lane, nx, hv);
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tfree[acc]);
        }
        if (!ok && lane == 0) atomicOr(err, 1);
    }
    __syncwarp();   // warp 0 reconverges after its MMA-issuing thread
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok && warp == 1) {   // let this CTA's copies in flight land before it exits
        if (nfill0) mbar_wait(&full[0], (uint32_t)((nfill0 - 1) & 1));
        if (nfill1) mbar_wait(&full[1], (uint32_t)((nfill1 - 1) & 1));
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(L1_TMEM_COLS)
                     : "memory");
    }
}

// Zero NC (multiple of 32) TMEM columns of this warp's lane quarter.
__device__ __forceinline__ void tmem_zero(uint32_t taddr, int nc) {
    const uint32_t z = 0u;
    for (int c = 0; c < nc; c += 32)
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
            "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};\n" ::"r"(taddr + (uint32_t)c),
            "r"(z)
            : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

// Stacked variant: one MMA per (staged input row j, dx, 16-channel step) with the weights of the
// five dy offsets stacked along N in reverse order, n = (4 - dy) CO + co, so that its 5 CO output
// columns land on the accumulators of output rows j - 4 .. j, which sit side by side when the
// accumulator of output row r starts at column (r + 4) CO.  Each staged A tile is read once for
// five offsets instead of once per offset; the accumulators of the 8 halo rows (r < 0, r >= R)
// collect unused sums, so every MMA accumulates onto zeroed tensor memory.
// in: [B][nz][ny][CI / 8][nx + 4][8] BF16, the padded channel-group layout (site x at x + 2, two
// periodic copies at each end), so that each staged row and channel group is one 2112-byte bulk
// (TMA) copy.  wt: [dz][dx][ci / 8][4 - dy][co][ci % 8].
// Persistent and warp-specialised: each CTA takes tiles (R output rows of 128 sites)
// blockIdx.x, + gridDim.x, ... and streams their planes (5 per tile):
//   warp 1 (copies)   loads each plane's weights into one of two buffers (`wfull` / `wfree`) and
//                     its R + 4 staged rows in four groups, a group refilled with the next plane's
//                     rows as soon as the MMAs that read it have completed (`afull` / `afree`);
//   thread 0 (MMAs)   issues a plane's MMAs group by group into one of NACC accumulator sets
//                     (alternating by tile) and commits `tfull` after a tile's last plane, once
//                     the epilogue has released that set (`tfree`);
//   warps 2..9        (two per TMEM lane quarter, half of the rows each) read a finished set,
//                     store the outputs, zero the set again and release it.
// EPI 0: tanh(acc + bias) -> BF16 in the padded layout (CO = 32); EPI 1: acc + bias -> FP32
// [site][16] (CO = 16) and the tile's FP64 sums of channels 0 and 1, added in a fixed order, into
// part[(b * 2 + c) * nblk + i] (i: the tile's index within its sample, nblk: tiles per sample).
constexpr int STK_THREADS = 320;

template <int CI, int CO, int EPI, int R, int NACC>
__global__ void __launch_bounds__(STK_THREADS, 1)
    k_conv_tc_stk(const bf16* __restrict__ in, const bf16* __restrict__ wt, const float* __restrict__ bias, int cout,
                  void* __restrict__ out, int nx, int ny, int nz, int B, double* __restrict__ part,
                  int* __restrict__ err) {
    constexpr int G = CI / 8;
    constexpr int ROWB = G * TC_XP * 16;
    constexpr int ABYTES = (R + 4) * ROWB;
    constexpr int NS = 5 * CO;                      // stacked N
    constexpr int WBYTES = 5 * G * NS * 16;         // weights of one dz
    constexpr int NGRP = 4;                         // row groups of a staged plane
    constexpr int RG = (R + 4) / NGRP;              // rows per group
    constexpr int NWB = 2;                          // weight buffers
    constexpr int SETC = (R + 8) * CO;              // TMEM columns of one accumulator set
    constexpr int TMEM_COLS = NACC * SETC;
    constexpr uint32_t IDESC = idesc_bf16(128, NS);
    static_assert(TMEM_COLS == 256 || TMEM_COLS == 512, "tensor-memory allocation");
    static_assert(NS % 16 == 0 && NS <= 256, "stacked N");
    static_assert(R % 2 == 0 && (R + 4) % NGRP == 0 && (SETC / 2) % 32 == 0, "R");
    static_assert(EPI != 0 || CO == 32, "the padded output layout holds 32 channels");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* As = smem;
    unsigned char* Ws = smem + ABYTES;
    __shared__ __align__(8) uint64_t afull[NGRP], afree[NGRP], wfull[NWB], wfree[NWB], tfull[NACC], tfree[NACC],
        psum[NACC];
    __shared__ uint32_t tmem_slot;
    __shared__ float csum[NACC][8][2];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nxt = nx / 128, nyb = ny / R;
    const int nblk = nz * nyb * nxt;   // tiles per sample
    const int ntile = B * nblk;
    const int nk = ntile > (int)blockIdx.x ? (ntile - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    const size_t V = (size_t)nx * ny * nz;
    auto tile_of = [&](int k, int& t, int& b, int& z, int& y0, int& x0) {
        t = (int)blockIdx.x + k * (int)gridDim.x;
        int u = t;
        x0 = (u % nxt) * 128;
        u /= nxt;
        y0 = (u % nyb) * R;
        u /= nyb;
        z = u % nz;
        b = u / nz;
    };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < NGRP; ++i) {
            mbar_init(&afull[i], 1);
            mbar_init(&afree[i], 1);
        }
        for (int i = 0; i < NWB; ++i) {
            mbar_init(&wfull[i], 1);
            mbar_init(&wfree[i], 1);
        }
        for (int i = 0; i < NACC; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tfree[i], 8);   // one arrival per epilogue warp
            mbar_init(&psum[i], 8);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const int q = warp & 3, half = (warp - 2) >> 2;   // epilogue warps: lane quarter, half of the rows
    const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
    if (warp >= 2)
        for (int a = 0; a < NACC; ++a) tmem_zero(tq + (uint32_t)(a * SETC + half * (SETC / 2)), SETC / 2);
    fence_before_sync();   // the zeroing precedes the first MMAs
    __syncthreads();
    fence_after_sync();

    bool ok = true;
    // planes whose weights / rows warp 1 has issued, and groups issued of the next plane's rows
    int nw_issued = 0, na_issued = 0, part_groups = 0;
    if (warp == 1) {   // bulk copies
        for (int P = 0; P < 5 * nk && ok; ++P) {
            int t, b, z, y0, x0;
            tile_of(P / 5, t, b, z, y0, x0);
            const int p = P % 5, wb = P % NWB;
            const int zin = wrapi_(z + p - 2, nz);
            const bf16* inb = in + (size_t)b * (V / nx) * G * (nx + 4) * 8;
            if (P >= NWB && !(ok = __all_sync(0xffffffffu, mbar_wait(&wfree[wb], (uint32_t)((P / NWB - 1) & 1)))))
                break;
            if (lane == 0) {
                mbar_expect(&wfull[wb], WBYTES);
                bulk_g2s(Ws + wb * WBYTES, wt + (size_t)p * (WBYTES / 2), WBYTES, &wfull[wb]);
            }
            nw_issued = P + 1;
            for (int gi = 0; gi < NGRP && ok; ++gi) {
                if (P >= 1 && !(ok = __all_sync(0xffffffffu, mbar_wait(&afree[gi], (uint32_t)((P - 1) & 1))))) break;
                if (lane == 0) mbar_expect(&afull[gi], RG * ROWB);
                __syncwarp();
                for (int c = lane; c < RG * G; c += 32) {
                    const int i = gi * RG + c / G, g = c % G;
                    const int yin = wrapi_(y0 - 2 + i, ny);
                    const bf16* src = inb + ((((size_t)zin * ny + yin) * G + g) * (nx + 4) + x0) * 8;
                    bulk_g2s(As + (i * G + g) * TC_XP * 16, src, TC_XP * 16, &afull[gi]);
                }
                part_groups = gi + 1;
            }
            if (ok) {
                na_issued = P + 1;
                part_groups = 0;
            }
        }
        if (!ok && lane == 0) atomicOr(err, 1);
    } else if (tid == 0) {   // MMA issue
        for (int k = 0; k < nk && ok; ++k) {
            const int acc = k % NACC;
            if (k >= NACC && !(ok = mbar_wait(&tfree[acc], (uint32_t)((k / NACC - 1) & 1)))) break;
            fence_after_sync();
            const uint32_t t0 = tmem + (uint32_t)(acc * SETC);
            for (int p = 0; p < 5 && ok; ++p) {
                const int P = 5 * k + p, wb = P % NWB;
                if (!(ok = mbar_wait(&wfull[wb], (uint32_t)((P / NWB) & 1)))) break;
                const uint32_t w0 = smem_u32(Ws + wb * WBYTES), a0 = smem_u32(As);
                for (int gi = 0; gi < NGRP; ++gi) {
                    if (!(ok = mbar_wait(&afull[gi], (uint32_t)(P & 1)))) break;
                    fence_after_sync();
                    for (int j = gi * RG; j < (gi + 1) * RG; ++j)
                        for (int dxi = 0; dxi < 5; ++dxi)
#pragma unroll
                            for (int kk = 0; kk < CI / 16; ++kk) {
                                const uint32_t aaddr = a0 + (uint32_t)((j * G + 2 * kk) * TC_XP + dxi) * 16u;
                                const uint32_t baddr = w0 + (uint32_t)((dxi * G + 2 * kk) * NS) * 16u;
                                mma_bf16(t0 + (uint32_t)(j * CO), smem_desc(aaddr, TC_XP * 16, 128),
                                         smem_desc(baddr, NS * 16, 128), IDESC, 1);
                            }
                    mma_commit(&afree[gi]);   // the group's rows may be refilled
                }
                if (ok) mma_commit(&wfree[wb]);   // the plane's weights may be overwritten
            }
            if (ok) mma_commit(&tfull[acc]);   // the tile's accumulators are complete
        }
        if (!ok) atomicOr(err, 1);
    } else if (warp >= 2) {   // epilogue
        float bs[CO];
#pragma unroll
        for (int co = 0; co < CO; ++co) bs[co] = co < cout ? bias[co] : 0.f;
        for (int k = 0; k < nk && ok; ++k) {
            const int acc = k % NACC;
            ok = __all_sync(0xffffffffu, mbar_wait(&tfull[acc], (uint32_t)((k / NACC) & 1)));
            if (!ok) break;
            fence_after_sync();
            int t, b, z, y0, x0;
            tile_of(k, t, b, z, y0, x0);
            const int x = x0 + q * 32 + lane;
            const uint32_t ts = tq + (uint32_t)(acc * SETC);
            float s0 = 0.f, s1 = 0.f;
#pragma unroll 1
            for (int r = half * (R / 2); r < (half + 1) * (R / 2); ++r) {
                float v[CO];
                const uint32_t col = (uint32_t)((r + 4) * CO);
                if (CO == 32) tmem_ld32(ts + col, v);
                else tmem_ld16(ts + col, v);
#pragma unroll
                for (int co = 0; co < CO; ++co) v[co] += bs[co];
                if (EPI == 0) {
                    __align__(16) bf16 hv[CO];
#pragma unroll
                    for (int co = 0; co < CO; ++co) hv[co] = __float2bfloat16(tanhf(v[co]));
                    store_padded32((bf16*)out, ((size_t)b * nz + z) * ny + y0 + r, x, nx, hv);
                } else {
                    const size_t site = (size_t)b * V + ((size_t)z * ny + (y0 + r)) * nx + x;
                    float4* dst = (float4*)((float*)out + site * 16);
#pragma unroll
                    for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    s0 += v[0];
                    s1 += v[1];
                }
            }
            tmem_zero(ts + (uint32_t)(half * (SETC / 2)), SETC / 2);   // ready for the set's next tile
            if (EPI == 1) {   // the tile's sums of the two output channels, in a fixed order
#pragma unroll
                for (int m = 16; m > 0; m >>= 1) {
                    s0 += __shfl_xor_sync(0xffffffffu, s0, m);
                    s1 += __shfl_xor_sync(0xffffffffu, s1, m);
                }
                if (lane == 0) {
                    csum[acc][warp - 2][0] = s0;
                    csum[acc][warp - 2][1] = s1;
                    mbar_arrive(&psum[acc]);
                }
                if (warp == 2) {
                    ok = __all_sync(0xffffffffu, mbar_wait(&psum[acc], (uint32_t)((k / NACC) & 1)));
                    if (ok && lane < 2) {
                        double sum = 0.0;
                        for (int w = 0; w < 8; ++w) sum += (double)csum[acc][w][lane];
                        part[((size_t)b * 2 + lane) * nblk + (t - b * nblk)] = sum;
                    }
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tfree[acc]);
        }
        if (!ok && lane == 0) atomicOr(err, 1);
    }
    __syncwarp();   // warp 0 reconverges after its MMA-issuing thread
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok && warp == 1) {   // copies in flight land before the CTA exits
        for (int i = 0; i < NWB && i < nw_issued; ++i) {
            const int last = nw_issued - 1 - ((nw_issued - 1 - i) % NWB);   // last plane loaded into buffer i
            mbar_wait(&wfull[i], (uint32_t)((last / NWB) & 1));
        }
        for (int gi = 0; gi < NGRP; ++gi) {
            const int n = na_issued + (gi < part_groups ? 1 : 0);
            if (n) mbar_wait(&afull[gi], (uint32_t)((n - 1) & 1));
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
    }
}

}  // namespace

// Bytes of dynamic shared memory of the first layer: two buffers of staged input rows and the
// weights of all 25 (dz, dy) offsets (every operand address its MMAs form lies inside them: the
// A walk ends at the last staged row of a buffer, the B walk at the last offset's weights).
size_t tc_conv_smem() { return (size_t)2 * L1_ABYTES + L1_WBYTES; }
// CTAs of a persistent layer: per_sm per SM, at most one per tile
int persist_grid(int ntile, int per_sm) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int g = (nsm > 0 ? nsm : 1) * per_sm;
    return ntile < g ? ntile : g;
}
// the stacked variant: R + 4 staged rows and NWB buffers of the weights of one whole dz
constexpr size_t stk_smem(int ci, int co, int r, int nwb) {
    return (size_t)(r + 4) * (ci / 8) * TC_XP * 16 + (size_t)nwb * 25 * (ci / 8) * co * 16;
}
constexpr int kR2 = 8, kR3 = 8;   // output rows per tile of the second and third layer
bool tc_conv_supported(int nx, int ny) { return nx % 128 == 0 && ny % kR2 == 0; }

int tc_conv_prepare() {
    // the whole unified L1/shared array as shared memory, so that several CTAs fit per SM
    cudaFuncSetAttribute(k_conv_tc_l1, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_conv_tc_stk<32, 32, 0, kR2, 1>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_conv_tc_stk<32, 16, 1, kR3, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaError_t e =
        cudaFuncSetAttribute(k_conv_tc_l1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_conv_smem());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_conv_tc_stk<32, 32, 0, kR2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)stk_smem(32, 32, kR2, 2));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_conv_tc_stk<32, 16, 1, kR3, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)stk_smem(32, 16, kR3, 2));
    return (int)e;
}

// CTAs per sample of the output layer (the number of its channel partial sums).
int tc_conv_blocks(int nx, int ny, int nz) { return nz * (ny / kR3) * (nx / 128); }

// Layer l of the predictor network (0: 2 -> 32 tanh with the x offsets folded into 16 input
// channels, input [B][nz][ny][2][nx + 4][8], weights [dz][dy][k / 8][co][k % 8]; 1: 32 -> 32 tanh
// and 2: 32 -> 16 linear FP32, both stacked, input [B][nz][ny][4][nx + 4][8], weights
// [dz][dx][ci / 8][4 - dy][co][ci % 8]) over B samples of an nx x ny x nz grid
// (tc_conv_supported must hold).  Persistent kernels: at most one CTA per tile.
void launch_conv_tc(int layer, const void* in, const void* wt, const float* bias, int cout, void* out, int nx, int ny,
                    int nz, int B, double* part, int* err, cudaStream_t s) {
    const bf16* x = (const bf16*)in;
    const bf16* w = (const bf16*)wt;
    if (layer == 0)
        k_conv_tc_l1<<<persist_grid(B * nz * (ny / TC_R) * (nx / 128), L1_CTAS_PER_SM), L1_THREADS, tc_conv_smem(),
                       s>>>(x, w, bias, cout, (bf16*)out, nx, ny, nz, B, err);
    else if (layer == 1)
        k_conv_tc_stk<32, 32, 0, kR2, 1><<<persist_grid(B * nz * (ny / kR2) * (nx / 128), 1), STK_THREADS,
                                           stk_smem(32, 32, kR2, 2), s>>>(x, w, bias, cout, out, nx, ny, nz, B, part, err);
    else
        k_conv_tc_stk<32, 16, 1, kR3, 2><<<persist_grid(B * nz * (ny / kR3) * (nx / 128), 1), STK_THREADS,
                                           stk_smem(32, 16, kR3, 2), s>>>(x, w, bias, cout, out, nx, ny, nz, B, part, err);
}

}  // namespace dscf
