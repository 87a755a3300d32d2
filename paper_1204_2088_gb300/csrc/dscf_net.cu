// Learned predictor of the density map: a translation-invariant 3-D convolution network
// phi_hat_I = phibar_I + y_I - <y_I>,  y = conv3(tanh(conv2(tanh(conv1(U - <U>))))),
// circular 5^3 kernels, 2 -> 32 -> 32 -> 2 channels (the paper has no such component; it stands
// in for the propagator solve inside the self-consistent inversion).
//
// Tensor cores: every convolution (forward, and backward with respect to the input) is one
// implicit GEMM over (offset, input channel) in BF16 with FP32 accumulation; weight gradients are
// per-offset GEMMs over sites.  The forward convolutions run on tcgen05 (operands in shared
// memory, accumulators in tensor memory; dscf_tc.cu) when nx is a multiple of 128 and ny of 8,
// and with warp-level mma.sync m16n8k16 otherwise (and for the backward pass).  Activations are stored
// channel-last in BF16 with channel counts padded to multiples of 16 (zero weights in the pad);
// the tcgen05 forward keeps its own copies in a padded channel-group layout (x16f, h1p, h2p) from
// which it stages rows by bulk copies, and the backward pass reads channel-last copies of them.
// Training keeps FP32 master weights and Adam moments.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/dscf.h"
#include "dscf_internal.cuh"

using namespace dscf;

namespace {

typedef __nv_bfloat16 bf16;

constexpr int NL = 3;
constexpr int KVOL = 125;
constexpr int CIN[NL] = {2, 32, 32}, COUT[NL] = {32, 32, 2};
constexpr int CINP[NL] = {16, 32, 32}, COUTP[NL] = {32, 32, 16};
constexpr size_t wcount(int l) { return (size_t)COUT[l] * CIN[l] * KVOL; }
constexpr size_t NPARAM = wcount(0) + 32 + wcount(1) + 32 + wcount(2) + 2;

enum { EPI_TANH = 0, EPI_LIN_F32 = 1, EPI_DTANH = 2 };

__device__ __forceinline__ int wrapd(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ unsigned ld32(const bf16* p) { return *(const unsigned*)p; }
__device__ __forceinline__ unsigned pack2(bf16 lo, bf16 hi) {
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}
__device__ __forceinline__ void mma16816(float* c, const unsigned* a, const unsigned* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Implicit-GEMM circular 5^3 convolution, one warp per 16 consecutive sites of an x row:
//   out[r][co] = sum_o sum_ci in[r + o][ci] W[o][co][ci]  (+ epilogue)
// in: [B][V][CI] bf16, W: [125][CO][CI] bf16.  Epilogues: tanh(acc + bias) -> bf16;
// acc + bias -> f32; acc * (1 - h^2) with h the forward activation -> bf16.
// With EPI_DTANH and bgrad != NULL, the FP32 values (before rounding to BF16) are also summed per
// channel into bgrad: the bias gradient of the layer whose activation is hact.
template <int CI, int CO, int EPI>
__global__ void __launch_bounds__(128) k_conv(const bf16* __restrict__ in, const bf16* __restrict__ W,
                                              const float* __restrict__ bias, int cout, const bf16* __restrict__ hact,
                                              void* __restrict__ out, int nx, int ny, int nz, int ntiles,
                                              float* __restrict__ bgrad) {
    const int lane = threadIdx.x & 31;
    const int mt = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (mt >= ntiles) return;
    const int V = nx * ny * nz;
    const int tpv = V / 16;
    const int b = mt / tpv;
    const int s0 = (mt - b * tpv) * 16;
    const int x0 = s0 % nx, y = (s0 / nx) % ny, z = s0 / (nx * ny);
    const int g = lane >> 2, t = lane & 3;
    const bf16* inb = in + (size_t)b * V * CI;
    float acc[CO / 8][4];
#pragma unroll
    for (int j = 0; j < CO / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (int o = 0; o < KVOL; ++o) {
        const int oz = o / 25 - 2, oy = (o / 5) % 5 - 2, ox = o % 5 - 2;
        const int rowoff = (wrapd(z + oz, nz) * ny + wrapd(y + oy, ny)) * nx;
        const int sa = rowoff + wrapd(x0 + g + ox, nx);       // site of A row g
        const int sb = rowoff + wrapd(x0 + g + 8 + ox, nx);   // site of A row g + 8
        const bf16* Wo = W + (size_t)o * CO * CI;
#pragma unroll
        for (int kc = 0; kc < CI / 16; ++kc) {
            unsigned a[4];
            const int c0 = kc * 16 + 2 * t;
            a[0] = ld32(inb + (size_t)sa * CI + c0);
            a[1] = ld32(inb + (size_t)sb * CI + c0);
            a[2] = ld32(inb + (size_t)sa * CI + c0 + 8);
            a[3] = ld32(inb + (size_t)sb * CI + c0 + 8);
#pragma unroll
            for (int j = 0; j < CO / 8; ++j) {
                unsigned bb[2];
                const bf16* wr = Wo + (size_t)(j * 8 + g) * CI + c0;
                bb[0] = ld32(wr);
                bb[1] = ld32(wr + 8);
                mma16816(acc[j], a, bb);
            }
        }
    }
    // epilogue: rows g, g + 8 (sites s0 + g, s0 + g + 8), columns co = 8 j + 2 t, +1
#pragma unroll
    for (int j = 0; j < CO / 8; ++j) {
        const int co = j * 8 + 2 * t;
        float bs0 = 0.f, bs1 = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const size_t site = (size_t)b * V + s0 + g + 8 * h;
            float v0 = acc[j][2 * h], v1 = acc[j][2 * h + 1];
            if (EPI == EPI_TANH || EPI == EPI_LIN_F32) {
                v0 += (co < cout) ? bias[co] : 0.f;
                v1 += (co + 1 < cout) ? bias[co + 1] : 0.f;
            }
            if (EPI == EPI_TANH) {
                v0 = tanhf(v0);
                v1 = tanhf(v1);
                *(unsigned*)((bf16*)out + site * CO + co) = pack2(__float2bfloat16(v0), __float2bfloat16(v1));
            } else if (EPI == EPI_LIN_F32) {
                *(float2*)((float*)out + site * CO + co) = make_float2(v0, v1);
            } else {
                const float h0 = __bfloat162float(hact[site * CO + co]), h1 = __bfloat162float(hact[site * CO + co + 1]);
                v0 *= 1.f - h0 * h0;
                v1 *= 1.f - h1 * h1;
                bs0 += v0;
                bs1 += v1;
                *(unsigned*)((bf16*)out + site * CO + co) = pack2(__float2bfloat16(v0), __float2bfloat16(v1));
            }
        }
        if (EPI == EPI_DTANH && bgrad) {   // sum over the 8 row groups (lane bits 2..4)
#pragma unroll
            for (int m = 4; m < 32; m <<= 1) {
                bs0 += __shfl_xor_sync(0xffffffffu, bs0, m);
                bs1 += __shfl_xor_sync(0xffffffffu, bs1, m);
            }
            if (g == 0) {
                if (co < cout) atomicAdd(&bgrad[co], bs0);
                if (co + 1 < cout) atomicAdd(&bgrad[co + 1], bs1);
            }
        }
    }
}

// Weight gradient of one layer: dW[co][ci][o] += sum_r in[r + o][ci] dout[r][co]; a GEMM per
// offset (M = input channels, N = output channels, K = sites) on tensor cores; each warp covers
// `chunk` consecutive m-tiles of sites and adds its FP32 partial with atomics.
template <int CI, int CO>
__global__ void __launch_bounds__(128) k_wgrad(const bf16* __restrict__ in, const bf16* __restrict__ dout,
                                               float* __restrict__ dW, int cin, int cout, int nx, int ny, int nz,
                                               int ntiles, int chunk) {
    const int lane = threadIdx.x & 31;
    const int o = blockIdx.y;
    const int w0 = (blockIdx.x * 4 + (threadIdx.x >> 5)) * chunk;
    const int g = lane >> 2, t = lane & 3;
    const int oz = o / 25 - 2, oy = (o / 5) % 5 - 2, ox = o % 5 - 2;
    const int V = nx * ny * nz;
    const int tpv = V / 16;
    float acc[CI / 16][CO / 8][4];
#pragma unroll
    for (int i = 0; i < CI / 16; ++i)
#pragma unroll
        for (int j = 0; j < CO / 8; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.f;
    for (int mt = w0; mt < min(w0 + chunk, ntiles); ++mt) {
        const int b = mt / tpv;
        const int s0 = (mt - b * tpv) * 16;
        const int x0 = s0 % nx, y = (s0 / nx) % ny, z = s0 / (nx * ny);
        const int rowoff = (wrapd(z + oz, nz) * ny + wrapd(y + oy, ny)) * nx;
        const bf16* inb = in + (size_t)b * V * CI;
        const bf16* db = dout + ((size_t)b * V + s0) * CO;
        // k index = site within the tile: pairs (2t, 2t+1) and (2t+8, 2t+9)
        int sk[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = 2 * t + (q & 1) + 8 * (q >> 1);
            sk[q] = rowoff + wrapd(x0 + k + ox, nx);
        }
#pragma unroll
        for (int i = 0; i < CI / 16; ++i) {
            unsigned a[4];
            const int ci0 = i * 16 + g;
            a[0] = pack2(inb[(size_t)sk[0] * CI + ci0], inb[(size_t)sk[1] * CI + ci0]);
            a[1] = pack2(inb[(size_t)sk[0] * CI + ci0 + 8], inb[(size_t)sk[1] * CI + ci0 + 8]);
            a[2] = pack2(inb[(size_t)sk[2] * CI + ci0], inb[(size_t)sk[3] * CI + ci0]);
            a[3] = pack2(inb[(size_t)sk[2] * CI + ci0 + 8], inb[(size_t)sk[3] * CI + ci0 + 8]);
#pragma unroll
            for (int j = 0; j < CO / 8; ++j) {
                const int co = j * 8 + g;
                unsigned bb[2];
                bb[0] = pack2(db[(size_t)(2 * t) * CO + co], db[(size_t)(2 * t + 1) * CO + co]);
                bb[1] = pack2(db[(size_t)(2 * t + 8) * CO + co], db[(size_t)(2 * t + 9) * CO + co]);
                mma16816(acc[i][j], a, bb);
            }
        }
    }
    // C rows = input channel (g, g + 8 within the m-tile), columns = output channel (2t, 2t+1)
#pragma unroll
    for (int i = 0; i < CI / 16; ++i)
#pragma unroll
        for (int j = 0; j < CO / 8; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int ci = i * 16 + g + 8 * (q >> 1);
                const int co = j * 8 + 2 * t + (q & 1);
                if (ci < cin && co < cout) atomicAdd(&dW[((size_t)co * cin + ci) * KVOL + o], acc[i][j][q]);
            }
}

// Per-sample, per-channel FP64 partial sums of a [B][C][V] float field (grid: blocks x C x B).
__global__ void k_chan_parts(const float* __restrict__ f, int C, int V, double* __restrict__ part) {
    __shared__ double sh[33];
    const int c = blockIdx.y, b = blockIdx.z;
    const float* p = f + ((size_t)b * C + c) * V;
    float acc = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) acc += p[i];
    const double t = block_sum((double)acc, sh);
    if (threadIdx.x == 0) part[((size_t)b * C + c) * gridDim.x + blockIdx.x] = t;
}
// Same for a channel-last [B][V][CS] float field (channels 0..C-1).
__global__ void k_chan_parts_cl(const float* __restrict__ f, int C, int CS, int V, double* __restrict__ part) {
    __shared__ double sh[33];
    const int c = blockIdx.y, b = blockIdx.z;
    const float* p = f + (size_t)b * V * CS + c;
    float acc = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) acc += p[(size_t)i * CS];
    const double t = block_sum((double)acc, sh);
    if (threadIdx.x == 0) part[((size_t)b * C + c) * gridDim.x + blockIdx.x] = t;
}
// means[p] = (sum of the nb partials of pair p, fixed order) / V, one block per pair.
__global__ void k_chan_final(const double* __restrict__ part, int nb, int V, double* __restrict__ means) {
    __shared__ double sh[33];
    const double* q = part + (size_t)blockIdx.x * nb;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += q[i];
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) means[blockIdx.x] = t / (double)V;
}

// Network input: x[r][c] = U_c[r] - <U_c> (c < 2), zero in the padded channels.
__global__ void k_net_in(const float* __restrict__ U, const double* __restrict__ means, int V, int B,
                         bf16* __restrict__ x) {
    const size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (r >= (size_t)B * V) return;
    const int b = (int)(r / V);
    const size_t i = r - (size_t)b * V;
    const float m0 = (float)means[2 * b], m1 = (float)means[2 * b + 1];
    __align__(16) bf16 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16(0.f);
    v[0] = __float2bfloat16(U[((size_t)2 * b) * V + i] - m0);
    v[1] = __float2bfloat16(U[((size_t)2 * b + 1) * V + i] - m1);
    uint4* dst = (uint4*)(x + r * 16);
    dst[0] = *(const uint4*)&v[0];
    dst[1] = *(const uint4*)&v[8];
}

// Network input with the five x offsets folded into the channels (tcgen05 first layer):
// xf[r][2 dx + c] = U_c[r + dx - 2 along x] - <U_c> for dx = 0..4, zero in channels 10..15, stored
// by channel group within each x row and with two periodic copies on each side of the row,
// [B][nz][ny][2][nx + 4][8] (site x at x + 2), so that a group's part of a tile's staged row,
// x0 - 2 .. x0 + 129, is one contiguous run.
__global__ void k_net_in_fold(const float* __restrict__ U, const double* __restrict__ means, int nx, int V, int B,
                              bf16* __restrict__ xf) {
    const size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (r >= (size_t)B * V) return;
    const int b = (int)(r / V);
    const int i = (int)(r - (size_t)b * V);
    const int x = i % nx, row = i - x;
    const float m0 = (float)means[2 * b], m1 = (float)means[2 * b + 1];
    const float* U0 = U + ((size_t)2 * b) * V + row;
    const float* U1 = U + ((size_t)2 * b + 1) * V + row;
    __align__(16) bf16 v[16];
#pragma unroll
    for (int dx = 0; dx < 5; ++dx) {
        int xs = x + dx - 2;
        xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
        v[2 * dx] = __float2bfloat16(U0[xs] - m0);
        v[2 * dx + 1] = __float2bfloat16(U1[xs] - m1);
    }
#pragma unroll
    for (int c = 10; c < 16; ++c) v[c] = __float2bfloat16(0.f);
    const size_t rowi = (size_t)b * (V / nx) + row / nx;
    bf16* g0 = xf + rowi * 2 * (size_t)(nx + 4) * 8;   // group 0 of this row; group 1 follows
    bf16* g1 = g0 + (size_t)(nx + 4) * 8;
    const int xp = x + 2;
    *(uint4*)(g0 + (size_t)xp * 8) = *(const uint4*)&v[0];
    *(uint4*)(g1 + (size_t)xp * 8) = *(const uint4*)&v[8];
    const int xh = x < 2 ? x + nx + 2 : (x >= nx - 2 ? x - nx + 2 : -1);   // periodic copy
    if (xh >= 0) {
        *(uint4*)(g0 + (size_t)xh * 8) = *(const uint4*)&v[0];
        *(uint4*)(g1 + (size_t)xh * 8) = *(const uint4*)&v[8];
    }
}

// Channel-last copy h[r][32] of an activation in the padded channel-group layout
// hp[rows][4][nx + 4][8] (site x at x + 2) that the tcgen05 forward writes; for the backward pass.
__global__ void k_unpad32(const bf16* __restrict__ hp, int nx, size_t S, bf16* __restrict__ h) {
    const size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (r >= S) return;
    const size_t rowi = r / nx;
    const int x = (int)(r - rowi * nx);
    const bf16* src = hp + (rowi * 4 * (size_t)(nx + 4) + (size_t)(x + 2)) * 8;
    uint4* dst = (uint4*)(h + r * 32);
#pragma unroll
    for (int g = 0; g < 4; ++g) dst[g] = *(const uint4*)(src + (size_t)g * (nx + 4) * 8);
}

// Network output: phi_c[r] = phibar_c + y[r][c] - <y_c>  ([B][2][V] float).
__global__ void k_net_out(const float* __restrict__ y, const double* __restrict__ means, int V, int B, double pb0,
                          double pb1, float* __restrict__ phi) {
    const size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (r >= (size_t)B * V) return;
    const int b = (int)(r / V);
    const size_t i = r - (size_t)b * V;
    const double m0 = means[2 * b], m1 = means[2 * b + 1];
    phi[((size_t)2 * b) * V + i] = (float)(pb0 - m0) + y[r * 16];
    phi[((size_t)2 * b + 1) * V + i] = (float)(pb1 - m1) + y[r * 16 + 1];
}

// Loss gradient: g = (phi - phi*) / n, projected mean-free per sample and channel (the output
// mean removal), written channel-last bf16 [B][V][16]; g is stored first in `gtmp` [B][2][V].
__global__ void k_loss_g(const float* __restrict__ phi, const float* __restrict__ tgt, size_t n, float* __restrict__ g,
                         double* __restrict__ lpart) {
    __shared__ double sh[33];
    float acc = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = phi[i] - tgt[i];
        g[i] = d / (float)n;
        acc += d * d;
    }
    const double t = block_sum((double)acc, sh);
    if (threadIdx.x == 0) lpart[blockIdx.x] = t;
}
__global__ void k_dy(const float* __restrict__ g, const double* __restrict__ means, int V, int B,
                     bf16* __restrict__ dy) {
    const size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (r >= (size_t)B * V) return;
    const int b = (int)(r / V);
    const size_t i = r - (size_t)b * V;
    const float m0 = (float)means[2 * b], m1 = (float)means[2 * b + 1];
    __align__(16) bf16 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16(0.f);
    v[0] = __float2bfloat16(g[((size_t)2 * b) * V + i] - m0);
    v[1] = __float2bfloat16(g[((size_t)2 * b + 1) * V + i] - m1);
    uint4* dst = (uint4*)(dy + r * 16);
    dst[0] = *(const uint4*)&v[0];
    dst[1] = *(const uint4*)&v[8];
}

// BF16 weight copies of layer l: forward Wf[o][co][ci] and input-gradient Wb[o'][ci][co] with
// Wb[o'][ci][co] = W[co][ci][-o'] (zero in padded channels).
__global__ void k_prep_w(const float* __restrict__ W, int cin, int cout, int cinp, int coutp, bf16* __restrict__ Wf,
                         bf16* __restrict__ Wb) {
    const int n = KVOL * coutp * cinp;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int o = i / (coutp * cinp), rem = i % (coutp * cinp);
        {
            const int co = rem / cinp, ci = rem % cinp;
            const float v = (co < cout && ci < cin) ? W[((size_t)co * cin + ci) * KVOL + o] : 0.f;
            Wf[i] = __float2bfloat16(v);
        }
        if (Wb) {
            const int ci = rem / coutp, co = rem % coutp;
            const int oz = o / 25 - 2, oy = (o / 5) % 5 - 2, ox = o % 5 - 2;
            const int of = (-oz + 2) * 25 + (-oy + 2) * 5 + (-ox + 2);
            const float v = (co < cout && ci < cin) ? W[((size_t)co * cin + ci) * KVOL + of] : 0.f;
            Wb[(size_t)o * cinp * coutp + (size_t)ci * coutp + co] = __float2bfloat16(v);
        }
    }
}

// BF16 weights of layer l in the tcgen05 operand layout Wt[o][ci / 8][co][ci % 8] (zero in
// padded channels): for each offset and group of 8 input channels, 8 output channels x 16 bytes
// form one contiguous core matrix.
__global__ void k_prep_wt(const float* __restrict__ W, int cin, int cout, int cinp, int coutp, bf16* __restrict__ Wt) {
    const int n = KVOL * coutp * cinp;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int o = i / (coutp * cinp), rem = i % (coutp * cinp);
        const int kc = rem / (coutp * 8), r2 = rem % (coutp * 8);
        const int co = r2 / 8, ci = kc * 8 + r2 % 8;
        const float v = (co < cout && ci < cin) ? W[((size_t)co * cin + ci) * KVOL + o] : 0.f;
        Wt[i] = __float2bfloat16(v);
    }
}

// Weights of a stacked tcgen05 layer: Wt[dz][dx][ci / 8][4 - dy][co][ci % 8] (zero in padded
// channels): per (dz, dx, 8 input channels) the five dy offsets' output channels, last dy first,
// form the rows of one N = 5 CO operand.
__global__ void k_prep_wt_stk(const float* __restrict__ W, int cin, int cout, int cinp, int coutp, bf16* __restrict__ Wt) {
    const int n = KVOL * coutp * cinp;
    const int G = cinp / 8;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int t = i;
        const int j8 = t % 8;
        t /= 8;
        const int co = t % coutp;
        t /= coutp;
        const int k = t % 5;
        t /= 5;
        const int kc = t % G;
        t /= G;
        const int dx = t % 5, dz = t / 5;
        const int ci = kc * 8 + j8, o = dz * 25 + (4 - k) * 5 + dx;
        const float v = (co < cout && ci < cin) ? W[((size_t)co * cin + ci) * KVOL + o] : 0.f;
        Wt[i] = __float2bfloat16(v);
    }
}

// First-layer weights for the folded input: Wt[dz][dy][k / 8][co][k % 8] with k = 2 dx + ci
// (k < 10), zero for k >= 10.
__global__ void k_prep_wt_fold(const float* __restrict__ W, bf16* __restrict__ Wt) {
    const int n = 25 * 2 * 32 * 8;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int o2 = i / 512, rem = i % 512;
        const int kc = rem / 256, r2 = rem % 256;
        const int co = r2 / 8, k = kc * 8 + r2 % 8;
        float v = 0.f;
        if (k < 10) v = W[((size_t)co * 2 + (k & 1)) * KVOL + o2 * 5 + (k >> 1)];
        Wt[i] = __float2bfloat16(v);
    }
}

// Adam (FP32 master weights).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct NetLayout {
    size_t params, grads, m, v, wf[NL], wb[NL], wt[NL], x16, x16f, h1, h2, h1p, h2p, y16, dy16, dz2, dz1, gtmp, part,
        means, lpart, err, bytes;
};
constexpr int kPartBlocks = 512;   // partial sums per channel and sample

NetLayout net_layout(int nx, int ny, int nz, int B) {
    NetLayout L;
    const size_t V = (size_t)nx * ny * nz, S = V * B;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = up256(off + bytes); return o; };
    L.params = take(NPARAM * 4);
    L.grads = take(NPARAM * 4);
    L.m = take(NPARAM * 4);
    L.v = take(NPARAM * 4);
    for (int l = 0; l < NL; ++l) {
        L.wf[l] = take((size_t)KVOL * COUTP[l] * CINP[l] * 2);
        L.wb[l] = take((size_t)KVOL * COUTP[l] * CINP[l] * 2);
        L.wt[l] = take((size_t)KVOL * COUTP[l] * CINP[l] * 2);
    }
    L.x16 = take(S * 16 * 2);
    L.x16f = tc_conv_supported(nx, ny) ? take(S / nx * (nx + 4) * 16 * 2) : 0;
    L.h1 = take(S * 32 * 2);
    L.h2 = take(S * 32 * 2);
    // the tcgen05 forward's activations, in the padded channel-group layout [rows][4][nx + 4][8]
    L.h1p = tc_conv_supported(nx, ny) ? take(S / nx * (nx + 4) * 32 * 2) : 0;
    L.h2p = tc_conv_supported(nx, ny) ? take(S / nx * (nx + 4) * 32 * 2) : 0;
    L.y16 = take(S * 16 * 4);
    L.dy16 = take(S * 16 * 2);
    L.dz2 = take(S * 32 * 2);
    L.dz1 = take(S * 32 * 2);
    L.gtmp = take(S * 2 * 4);
    const size_t ntc = tc_conv_supported(nx, ny) ? (size_t)tc_conv_blocks(nx, ny, nz) : 0;
    L.part = take((size_t)B * 2 * (ntc > (size_t)kPartBlocks ? ntc : (size_t)kPartBlocks) * 8);
    L.means = take((size_t)B * 2 * 8);
    L.lpart = take((size_t)1024 * 8);
    L.err = take(sizeof(int));
    L.bytes = off;
    return L;
}

size_t poff(int l) {   // offset of layer l's weights in the parameter vector (bias follows)
    size_t o = 0;
    for (int k = 0; k < l; ++k) o += wcount(k) + COUT[k];
    return o;
}

thread_local std::string g_net_err;

}  // namespace

struct dscf_net {
    int nx, ny, nz, B, device;
    size_t V;
    cudaStream_t stream;
    char* ws;
    NetLayout L;
    int adam_t = 0;
    int path = 0;          // 0: tcgen05 forward where the grid allows it, 1: mma.sync only
    bool tc_ok = false;    // grid and device allow the tcgen05 forward
    std::string err;
    bool use_tc() const { return tc_ok && path == 0; }
    template <typename P> P* at(size_t off) { return (P*)(ws + off); }
};

namespace {

int nfail(dscf_net* n, int code, const char* msg) {
    if (n) n->err = msg; else g_net_err = msg;
    return code;
}
int ncheck(dscf_net* n, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return DSCF_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return nfail(n, DSCF_ERR_CUDA, m.c_str());
}

void prep_weights(dscf_net* n) {
    for (int l = 0; l < NL; ++l)
        k_prep_w<<<64, 256, 0, n->stream>>>(n->at<float>(n->L.params) + poff(l), CIN[l], COUT[l], CINP[l], COUTP[l],
                                              n->at<bf16>(n->L.wf[l]), l > 0 ? n->at<bf16>(n->L.wb[l]) : nullptr);
    if (n->tc_ok) {
        k_prep_wt_fold<<<64, 256, 0, n->stream>>>(n->at<float>(n->L.params) + poff(0), n->at<bf16>(n->L.wt[0]));
        for (int l = 1; l < NL; ++l)
            k_prep_wt_stk<<<64, 256, 0, n->stream>>>(n->at<float>(n->L.params) + poff(l), CIN[l], COUT[l], CINP[l],
                                                       COUTP[l], n->at<bf16>(n->L.wt[l]));
    }
}

// means of C = 2 channels of a [B][C][V] field into L.means
void chan_means(dscf_net* n, const float* f, int C) {
    k_chan_parts<<<dim3(kPartBlocks, C, n->B), 256, 0, n->stream>>>(f, C, (int)n->V, n->at<double>(n->L.part));
    k_chan_final<<<C * n->B, 256, 0, n->stream>>>(n->at<double>(n->L.part), kPartBlocks, (int)n->V,
                                                  n->at<double>(n->L.means));
}

// forward pass from U ([B][2][V] float, device) to phi ([B][2][V] float, device)
void forward(dscf_net* n, const float* U, double pb0, double pb1, float* phi) {
    const int V = (int)n->V, B = n->B;
    const int ntiles = (int)(n->V * B / 16);
    const int blocks = (ntiles + 3) / 4;
    const int eb = (int)((n->V * B + 255) / 256);
    chan_means(n, U, 2);
    k_net_in<<<eb, 256, 0, n->stream>>>(U, n->at<double>(n->L.means), V, B, n->at<bf16>(n->L.x16));
    if (n->use_tc()) {
        k_net_in_fold<<<eb, 256, 0, n->stream>>>(U, n->at<double>(n->L.means), n->nx, V, B, n->at<bf16>(n->L.x16f));
        const size_t act[NL + 1] = {n->L.x16f, n->L.h1p, n->L.h2p, n->L.y16};
        for (int l = 0; l < NL; ++l)
            launch_conv_tc(l, n->ws + act[l], n->ws + n->L.wt[l], n->at<float>(n->L.params) + poff(l) + wcount(l),
                           COUT[l], n->ws + act[l + 1], n->nx, n->ny, n->nz, B, n->at<double>(n->L.part),
                           n->at<int>(n->L.err), n->stream);
        // the output layer left per-CTA sums of its two channels
        k_chan_final<<<2 * B, 256, 0, n->stream>>>(n->at<double>(n->L.part), tc_conv_blocks(n->nx, n->ny, n->nz), V,
                                                   n->at<double>(n->L.means));
    } else {
        k_conv<16, 32, EPI_TANH><<<blocks, 128, 0, n->stream>>>(n->at<bf16>(n->L.x16), n->at<bf16>(n->L.wf[0]),
            n->at<float>(n->L.params) + poff(0) + wcount(0), 32, nullptr, n->at<bf16>(n->L.h1), n->nx, n->ny, n->nz, ntiles,
            nullptr);
        k_conv<32, 32, EPI_TANH><<<blocks, 128, 0, n->stream>>>(n->at<bf16>(n->L.h1), n->at<bf16>(n->L.wf[1]),
            n->at<float>(n->L.params) + poff(1) + wcount(1), 32, nullptr, n->at<bf16>(n->L.h2), n->nx, n->ny, n->nz, ntiles,
            nullptr);
        k_conv<32, 16, EPI_LIN_F32><<<blocks, 128, 0, n->stream>>>(n->at<bf16>(n->L.h2), n->at<bf16>(n->L.wf[2]),
            n->at<float>(n->L.params) + poff(2) + wcount(2), 2, nullptr, n->at<float>(n->L.y16), n->nx, n->ny, n->nz, ntiles,
            nullptr);
        k_chan_parts_cl<<<dim3(kPartBlocks, 2, B), 256, 0, n->stream>>>(n->at<float>(n->L.y16), 2, 16, V,
                                                                         n->at<double>(n->L.part));
        k_chan_final<<<2 * B, 256, 0, n->stream>>>(n->at<double>(n->L.part), kPartBlocks, V, n->at<double>(n->L.means));
    }
    k_net_out<<<eb, 256, 0, n->stream>>>(n->at<float>(n->L.y16), n->at<double>(n->L.means), V, B, pb0, pb1, phi);
}

// gradient of 0.5 mean((phi - target)^2) with respect to all parameters, into grads
void backward(dscf_net* n, const float* phi, const float* tgt) {
    const int V = (int)n->V, B = n->B;
    const size_t S = n->V * B;
    const int ntiles = (int)(S / 16);
    const int blocks = (ntiles + 3) / 4;
    const int eb = (int)((S + 255) / 256);
    float* grads = n->at<float>(n->L.grads);
    if (n->use_tc()) {   // the forward pass left its activations in the padded layout
        k_unpad32<<<eb, 256, 0, n->stream>>>(n->at<bf16>(n->L.h1p), n->nx, S, n->at<bf16>(n->L.h1));
        k_unpad32<<<eb, 256, 0, n->stream>>>(n->at<bf16>(n->L.h2p), n->nx, S, n->at<bf16>(n->L.h2));
    }
    cudaMemsetAsync(grads, 0, NPARAM * 4, n->stream);
    k_loss_g<<<1024, 256, 0, n->stream>>>(phi, tgt, S * 2, n->at<float>(n->L.gtmp), n->at<double>(n->L.lpart));
    chan_means(n, n->at<float>(n->L.gtmp), 2);
    k_dy<<<eb, 256, 0, n->stream>>>(n->at<float>(n->L.gtmp), n->at<double>(n->L.means), V, B, n->at<bf16>(n->L.dy16));
    const int chunk = 8;
    const int wblocks = (ntiles + 4 * chunk - 1) / (4 * chunk);
    // layer 3
    k_wgrad<32, 16><<<dim3(wblocks, KVOL), 128, 0, n->stream>>>(n->at<bf16>(n->L.h2), n->at<bf16>(n->L.dy16),
        grads + poff(2), 32, 2, n->nx, n->ny, n->nz, ntiles, chunk);
    // the output bias cannot change phi_hat (its per-sample mean is removed): its gradient is zero
    k_conv<16, 32, EPI_DTANH><<<blocks, 128, 0, n->stream>>>(n->at<bf16>(n->L.dy16), n->at<bf16>(n->L.wb[2]), nullptr,
        32, n->at<bf16>(n->L.h2), n->at<bf16>(n->L.dz2), n->nx, n->ny, n->nz, ntiles, grads + poff(1) + wcount(1));
    // layer 2
    k_wgrad<32, 32><<<dim3(wblocks, KVOL), 128, 0, n->stream>>>(n->at<bf16>(n->L.h1), n->at<bf16>(n->L.dz2),
        grads + poff(1), 32, 32, n->nx, n->ny, n->nz, ntiles, chunk);
    k_conv<32, 32, EPI_DTANH><<<blocks, 128, 0, n->stream>>>(n->at<bf16>(n->L.dz2), n->at<bf16>(n->L.wb[1]), nullptr,
        32, n->at<bf16>(n->L.h1), n->at<bf16>(n->L.dz1), n->nx, n->ny, n->nz, ntiles, grads + poff(0) + wcount(0));
    // layer 1
    k_wgrad<16, 32><<<dim3(wblocks, KVOL), 128, 0, n->stream>>>(n->at<bf16>(n->L.x16), n->at<bf16>(n->L.dz1),
        grads + poff(0), 2, 32, n->nx, n->ny, n->nz, ntiles, chunk);
}

// splitmix64-based normal deviates for the initial weights (Box-Muller)
double u01(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

}  // namespace

bool dscf_net_fits(const dscf_net* n, int nx, int ny, int nz) {
    return n && n->nx == nx && n->ny == ny && n->nz == nz && n->B == 1;
}
int dscf_net_forward_launches(const dscf_net* n) { return 9; }
void dscf_net_forward_on(dscf_net* n, cudaStream_t stream, const float* U, double pb0, double pb1, float* phi) {
    cudaStream_t keep = n->stream;
    n->stream = stream;
    forward(n, U, pb0, pb1, phi);
    n->stream = keep;
}

extern "C" {

size_t dscf_net_workspace_bytes(int32_t nx, int32_t ny, int32_t nz, int32_t batch) {
    if (nx < 16 || nx % 16 || ny < 1 || nz < 1 || batch < 1) return 0;
    return net_layout(nx, ny, nz, batch).bytes;
}

int dscf_net_init(int32_t nx, int32_t ny, int32_t nz, int32_t batch, uint64_t seed, void* workspace, size_t bytes,
                  void* stream, dscf_net** out) {
    if (!out) return nfail(nullptr, DSCF_ERR_ARG, "out is NULL");
    *out = nullptr;
    const size_t need = dscf_net_workspace_bytes(nx, ny, nz, batch);
    if (need == 0) return nfail(nullptr, DSCF_ERR_ARG, "need nx a multiple of 16, ny, nz, batch >= 1");
    if (!workspace || ((uintptr_t)workspace & 255)) return nfail(nullptr, DSCF_ERR_ARG, "workspace must be 256-byte aligned");
    if (bytes < need) return nfail(nullptr, DSCF_ERR_OOM, "workspace too small");
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, workspace) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return nfail(nullptr, DSCF_ERR_ARG, "workspace is not device memory");
    }
    dscf_net* n = new (std::nothrow) dscf_net;
    if (!n) return nfail(nullptr, DSCF_ERR_OOM, "host allocation failed");
    n->nx = nx; n->ny = ny; n->nz = nz; n->B = batch; n->device = pa.device;
    n->V = (size_t)nx * ny * nz;
    n->stream = (cudaStream_t)stream;
    n->ws = (char*)workspace;
    n->L = net_layout(nx, ny, nz, batch);
    cudaSetDevice(n->device);
    {
        int major = 0, minor = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, n->device);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, n->device);
        n->tc_ok = tc_conv_supported(nx, ny) && major == 10 && minor == 3 && tc_conv_prepare() == 0;
        cudaGetLastError();
    }
    // Glorot-like normal initial weights, zero biases
    std::vector<float> p(NPARAM, 0.f);
    uint64_t k = 0;
    for (int l = 0; l < NL; ++l) {
        const double sd = std::sqrt(2.0 / ((double)(CIN[l] + COUT[l]) * KVOL));
        float* w = p.data() + poff(l);
        for (size_t i = 0; i < wcount(l); ++i, k += 2) {
            const double u1 = 1.0 - u01(seed, k), u2 = u01(seed, k + 1);
            w[i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    }
    int rc = ncheck(n, cudaMemcpy(n->at<float>(n->L.params), p.data(), NPARAM * 4, cudaMemcpyHostToDevice), "params");
    if (!rc) rc = ncheck(n, cudaMemset(n->at<float>(n->L.m), 0, NPARAM * 4), "m");
    if (!rc) rc = ncheck(n, cudaMemset(n->at<float>(n->L.v), 0, NPARAM * 4), "v");
    if (!rc) rc = ncheck(n, cudaMemset(n->at<int>(n->L.err), 0, sizeof(int)), "error word");
    if (!rc) {
        prep_weights(n);
        rc = ncheck(n, cudaStreamSynchronize(n->stream), "init");
    }
    if (rc) { g_net_err = n->err; delete n; return rc; }
    *out = n;
    return DSCF_OK;
}

int dscf_net_forward(dscf_net* n, const float* U, const double* phibar, float* phi_out) {
    if (!n || !U || !phibar || !phi_out) return n ? nfail(n, DSCF_ERR_ARG, "NULL argument") : DSCF_ERR_ARG;
    cudaSetDevice(n->device);
    forward(n, U, phibar[0], phibar[1], phi_out);
    return ncheck(n, cudaGetLastError(), "net forward");
}

int dscf_net_gradient(dscf_net* n, const float* U, const float* phi_target, const double* phibar, float* phi_work,
                      double* loss, float* grads_out) {
    if (!n || !U || !phi_target || !phibar || !phi_work) return n ? nfail(n, DSCF_ERR_ARG, "NULL argument") : DSCF_ERR_ARG;
    cudaSetDevice(n->device);
    forward(n, U, phibar[0], phibar[1], phi_work);
    backward(n, phi_work, phi_target);
    int rc = ncheck(n, cudaGetLastError(), "net gradient");
    if (rc) return rc;
    if (loss) {
        std::vector<double> lp(1024);
        rc = ncheck(n, cudaMemcpyAsync(lp.data(), n->at<double>(n->L.lpart), 1024 * 8, cudaMemcpyDeviceToHost, n->stream),
                    "loss");
        if (!rc) rc = ncheck(n, cudaStreamSynchronize(n->stream), "loss sync");
        if (rc) return rc;
        double s = 0.0;
        for (double v : lp) s += v;
        *loss = 0.5 * s / (double)(n->V * n->B * 2);
    }
    if (grads_out)
        return ncheck(n, cudaMemcpyAsync(grads_out, n->at<float>(n->L.grads), NPARAM * 4, cudaMemcpyDeviceToDevice, n->stream),
                      "grads");
    return DSCF_OK;
}

int dscf_net_train_step(dscf_net* n, const float* U, const float* phi_target, const double* phibar, float* phi_work,
                        float lr, double* loss) {
    int rc = dscf_net_gradient(n, U, phi_target, phibar, phi_work, loss, nullptr);
    if (rc) return rc;
    n->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)n->adam_t), c2 = 1.f - std::pow(b2, (float)n->adam_t);
    k_adam<<<256, 256, 0, n->stream>>>(n->at<float>(n->L.params), n->at<float>(n->L.grads), n->at<float>(n->L.m),
                                       n->at<float>(n->L.v), (int)NPARAM, lr, b1, b2, 1e-8f, c1, c2);
    prep_weights(n);
    return ncheck(n, cudaGetLastError(), "adam");
}

int dscf_net_get_params(dscf_net* n, float* dst) {
    if (!n || !dst) return DSCF_ERR_ARG;
    return ncheck(n, cudaMemcpyAsync(dst, n->at<float>(n->L.params), NPARAM * 4, cudaMemcpyDefault, n->stream), "get params");
}

int dscf_net_set_params(dscf_net* n, const float* src) {
    if (!n || !src) return DSCF_ERR_ARG;
    int rc = ncheck(n, cudaMemcpyAsync(n->at<float>(n->L.params), src, NPARAM * 4, cudaMemcpyDefault, n->stream), "set params");
    if (rc) return rc;
    prep_weights(n);
    n->adam_t = 0;
    cudaMemsetAsync(n->at<float>(n->L.m), 0, NPARAM * 4, n->stream);
    cudaMemsetAsync(n->at<float>(n->L.v), 0, NPARAM * 4, n->stream);
    return ncheck(n, cudaGetLastError(), "set params");
}

int64_t dscf_net_num_params(void) { return (int64_t)NPARAM; }

int dscf_net_set_tensor_path(dscf_net* n, int32_t path) {
    if (!n) return DSCF_ERR_ARG;
    if (path != 0 && path != 1) return nfail(n, DSCF_ERR_ARG, "path must be 0 (tcgen05 where possible) or 1 (mma.sync)");
    cudaSetDevice(n->device);
    int rc = ncheck(n, cudaStreamSynchronize(n->stream), "path sync");
    if (rc) return rc;
    n->path = path;
    return DSCF_OK;
}

int32_t dscf_net_tensor_path(const dscf_net* n) { return n ? (n->use_tc() ? 2 : 1) : 0; }

int dscf_net_status(dscf_net* n) {
    if (!n) return DSCF_ERR_ARG;
    cudaSetDevice(n->device);
    int e = 0;
    int rc = ncheck(n, cudaStreamSynchronize(n->stream), "status sync");
    if (!rc) rc = ncheck(n, cudaMemcpy(&e, n->at<int>(n->L.err), sizeof(int), cudaMemcpyDeviceToHost), "status read");
    if (rc) return rc;
    if (e) {
        cudaMemset(n->at<int>(n->L.err), 0, sizeof(int));
        return nfail(n, DSCF_ERR_TIMEOUT, "a tensor-core convolution gave up waiting for its MMAs");
    }
    return DSCF_OK;
}

int dscf_net_free(dscf_net* n) {
    delete n;
    return DSCF_OK;
}

const char* dscf_net_last_error(const dscf_net* n) { return n ? n->err.c_str() : g_net_err.c_str(); }

}  // extern "C"
