// Forward density map phi[U] without any device allocation by the caller or the library.
//
// Some callers cannot call cudaMalloc (or any allocator) at all: code running inside a host
// framework that owns every device allocation and hands out only its own buffers, plug-ins
// invoked from a callback where allocation is forbidden, or processes that must not grow their
// device footprint after start-up.  They cannot provide the workspace the context-based API
// needs.  This entry point takes only the input potentials and the output densities; the
// propagator stack, Boltzmann factors, quadratures, partial sums and replica table live in one
// file-scope device array of fixed size, which every GPU that loads this code keeps for the life
// of the process.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/dscf.h"
#include "dscf_internal.cuh"

using namespace dscf;

namespace dscf {
void set_thread_error(const char* msg);
}

namespace {

static __device__ __align__(256) unsigned char g_scratch[DSCF_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_dev[kMaxDevices] = {};   // device address of g_scratch, per device

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Writes the replica descriptor into the scratch; passed by value so no host-to-device copy
// (and no staging buffer) is needed.
__global__ void k_put_rep(Rep* dst, Rep r) { *dst = r; }

}  // namespace

namespace {
int densities_static_on(const dscf_params* p, int32_t precision, const void* U_in, void* phi_out, void* stream);
}

// Runs on the device that holds U_in and leaves the calling thread's current device as it found it.
extern "C" int dscf_densities_static(const dscf_params* p, int32_t precision, const void* U_in, void* phi_out,
                                     void* stream) {
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        cudaGetLastError();
        set_thread_error("dscf_densities_static: cudaGetDevice failed");
        return DSCF_ERR_CUDA;
    }
    const int rc = densities_static_on(p, precision, U_in, phi_out, stream);
    if (cudaSetDevice(prev) != cudaSuccess && rc == DSCF_OK) {
        set_thread_error("dscf_densities_static: restoring the caller's device failed");
        return DSCF_ERR_CUDA;
    }
    return rc;
}

namespace {
int densities_static_on(const dscf_params* p, int32_t precision, const void* U_in, void* phi_out, void* stream) {
    if (!p || !U_in || !phi_out) {
        set_thread_error("dscf_densities_static: NULL argument");
        return DSCF_ERR_ARG;
    }
    if (precision != DSCF_FP64 && precision != DSCF_FP32) {
        set_thread_error("dscf_densities_static: bad precision");
        return DSCF_ERR_ARG;
    }
    if (dscf_workspace_bytes(p, 1, precision) == 0) {
        set_thread_error("dscf_densities_static: invalid parameters");
        return DSCF_ERR_ARG;
    }
    // the device that holds the input selects the copy of the scratch array
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, U_in) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        set_thread_error("dscf_densities_static: U_in is not device memory");
        return DSCF_ERR_ARG;
    }
    const int dev = pa.device;
    if (dev < 0 || dev >= kMaxDevices) {
        set_thread_error("dscf_densities_static: device index out of range");
        return DSCF_ERR_ARG;
    }
    if (cudaSetDevice(dev) != cudaSuccess) {
        set_thread_error("dscf_densities_static: cudaSetDevice failed");
        return DSCF_ERR_CUDA;
    }

    // Tiling of one replica, as the context-based path does it.
    const size_t es = precision == DSCF_FP64 ? sizeof(double) : sizeof(float);
    Rep R;
    std::memset(&R, 0, sizeof R);
    R.nx = p->nx; R.ny = p->ny; R.nz = p->nz; R.ns = p->ns; R.N = p->N; R.nA = p->nA;
    R.V = (long long)p->nx * p->ny * p->nz;
    tile_replica(R, 8);
    R.phi_p = p->phi_p;
    R.alpha = p->a * p->a / 6.0;
    R.part_stride = R.ntiles > R.nblk ? R.ntiles : R.nblk;

    // Scratch layout: replica table, maps, Boltzmann factors, propagators, quadratures,
    // partial sums, scalars.
    const size_t V = (size_t)R.V;
    size_t off = 0;
    const size_t o_rep = off; off = up256(off + sizeof(Rep));
    const size_t o_t2r = off; off = up256(off + sizeof(int) * R.ntiles);
    const size_t o_b2r = off; off = up256(off + sizeof(int) * R.nblk);
    const size_t o_E = off; off = up256(off + (size_t)R.ns * V * es);
    const size_t o_G = off; off = up256(off + (size_t)R.N * V * es);
    const size_t o_Gp0 = off; off = up256(off + V * es);
    const size_t o_Gp1 = off; off = up256(off + V * es);
    const size_t o_q = off; off = up256(off + 2 * V * es);
    const size_t o_part = off; off = up256(off + sizeof(double) * NPART * (size_t)R.part_stride);
    const size_t o_scal = off; off = up256(off + sizeof(double) * kScalStride);
    if (off > (size_t)DSCF_STATIC_SCRATCH_BYTES) {
        set_thread_error("dscf_densities_static: the problem needs more scratch than DSCF_STATIC_SCRATCH_BYTES");
        return DSCF_ERR_OOM;
    }

    // Set-up, once per device: the host-side name g_scratch is only a stand-in, the kernels need
    // the device address of this device's copy.
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_dev[dev]) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess || !ptr) {
                set_thread_error("dscf_densities_static: cudaGetSymbolAddress failed");
                return DSCF_ERR_CUDA;
            }
            g_scratch_dev[dev] = (unsigned char*)ptr;
            // dynamic shared memory of the propagator kernels, for the largest layout
            if (prop_set_smem_limit<double>(prop_smem_bytes(4, true, 8)) != 0 ||
                prop_set_smem_limit<float>(prop_smem_bytes(4, true, 4)) != 0) {
                g_scratch_dev[dev] = nullptr;
                set_thread_error("dscf_densities_static: cudaFuncSetAttribute failed");
                return DSCF_ERR_CUDA;
            }
        }
        base = g_scratch_dev[dev];
    }
    R.E = base + o_E;
    R.G = base + o_G;
    R.Gp0 = base + o_Gp0;
    R.Gp1 = base + o_Gp1;
    R.q = base + o_q;
    R.part = (double*)(base + o_part);
    R.scal = (double*)(base + o_scal);
    R.tile0 = 0;
    R.blk0 = 0;
    R.ext_off = 0;
    R.vbase = 0;

    cudaStream_t s = (cudaStream_t)stream;
    Launch L;
    L.reps = (const Rep*)(base + o_rep);
    L.tile2rep = (const int*)(base + o_t2r);
    L.blk2rep = (const int*)(base + o_b2r);
    L.status = nullptr;
    L.counter = nullptr;
    L.nblk_total = R.nblk;
    L.nlb_total = R.lb_nblk;
    L.nrep = 1;
    L.stream = s;
    // the only state that must start at zero: the tile and block maps (one replica, index 0)
    cudaError_t e = cudaMemsetAsync(base + o_t2r, 0, sizeof(int) * R.ntiles, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_b2r, 0, sizeof(int) * R.nblk, s);
    if (e != cudaSuccess) {
        set_thread_error("dscf_densities_static: cudaMemsetAsync failed");
        return DSCF_ERR_CUDA;
    }
    k_put_rep<<<1, 1, 0, s>>>((Rep*)(base + o_rep), R);
    if (precision == DSCF_FP64) {
        launch_exp<double>(L, 3, 0, U_in);
        for (int k = 1; k <= R.N; ++k) launch_prop_fwd<double>(L, k, R.ntiles, prop_smem_bytes(R.vec, false, 8));
        for (int j = 0; j < R.N; ++j) launch_prop_bwd<double>(L, j, R.ntiles, prop_smem_bytes(R.vec, true, 8));
        launch_dens_out<double>(L, phi_out);
    } else {
        launch_exp<float>(L, 3, 0, U_in);
        for (int k = 1; k <= R.N; ++k) launch_prop_fwd<float>(L, k, R.ntiles, prop_smem_bytes(R.vec, false, 4));
        for (int j = 0; j < R.N; ++j) launch_prop_bwd<float>(L, j, R.ntiles, prop_smem_bytes(R.vec, true, 4));
        launch_dens_out<float>(L, phi_out);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_thread_error(cudaGetErrorString(e));
        return DSCF_ERR_CUDA;
    }
    return DSCF_OK;
}
}  // namespace
