// Physics step for callers that cannot allocate device memory.
//
// Some callers run where device allocation is not available to them: code
// executing inside a captured CUDA graph region they do not own, plug-ins
// handed a fixed device arena by a host application, or processes whose
// allocator is owned by another runtime.  vuda_sim_step_noalloc serves them:
// the caller passes every input and output as device memory it already
// owns, and the only scratch the step needs -- the per-environment offsets
// of the contact spill area and the spill records themselves (contacts that
// do not fit the kernel's shared-memory records) -- lives in one file-scope
// device array of fixed size, allocated when the library is loaded on a
// device and held until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.cuh"

namespace vuda {
namespace {

// Scratch capacity in 4-byte words: 16 MiB.  The first (E + 1) * 2 words hold
// the int64 spill offsets, the rest holds spill records of kContactStride
// words, max_contacts_per_body per body.
constexpr size_t kNoAllocWords = 4u << 20;

__device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

// Per-device address of the scratch array, resolved once with that device
// current.  A host-side reference to g_noalloc_scratch names a host stand-in,
// never the device memory, so the address must come from the runtime.
struct ScratchAddr {
    void* ptr[64] = {};
    std::mutex mu;
};
ScratchAddr& scratch_addr() {
    static ScratchAddr s;
    return s;
}

__global__ void spill_offsets_kernel(const int32_t* __restrict__ body_off, int E, int mcpb, int64_t* off) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e <= E) off[e] = (int64_t)mcpb * body_off[e];
}

}  // namespace
}  // namespace vuda

using namespace vuda;

extern "C" vuda_status vuda_sim_step_noalloc(int32_t num_envs, int32_t num_bodies, int32_t max_bodies,
                                             const int32_t* body_off, float* pos, float* quat, float* vel,
                                             float* angvel, const uint8_t* shape_type, const float* shape_dims,
                                             const float* inv_mass, const float* inv_inertia, const float* force,
                                             const vuda_sim_params* prm, int32_t nsteps, float* pose,
                                             uint32_t* flags, int32_t* ncontacts, int32_t smem_per_env,
                                             vuda_stream_t stream) {
    if (!prm || num_envs < 0 || num_bodies < 0 || max_bodies < 0 || nsteps < 0) {
        set_error("vuda_sim_step_noalloc: bad argument");
        return VUDA_ERR_INVALID;
    }
    if (prm->substeps <= 0 || prm->iterations < 0 || prm->max_contacts_per_body <= 0 || !(prm->dt > 0.0f)) {
        set_error("vuda_sim_step_noalloc: bad sim params");
        return VUDA_ERR_INVALID;
    }
    if (num_envs > 0 && max_bodies <= 0) {
        set_error("vuda_sim_step_noalloc: max_bodies must be positive");
        return VUDA_ERR_INVALID;
    }
    if (prm->hull_contacts) {
        set_error("vuda_sim_step_noalloc: hull contacts need the batch's meshes (vuda_env_create)");
        return VUDA_ERR_INVALID;
    }
    if (num_envs == 0 || nsteps == 0) return VUDA_OK;
    if (!body_off || !pos || !quat || !vel || !angvel || !shape_type || !shape_dims || !inv_mass || !inv_inertia ||
        !pose || !flags || !ncontacts) {
        set_error("vuda_sim_step_noalloc: null device array");
        return VUDA_ERR_INVALID;
    }
    if ((int64_t)prm->max_contacts_per_body * max_bodies > 32767) {
        set_error("vuda_sim_step_noalloc: max_contacts_per_body * max_bodies must stay below 32768");
        return VUDA_ERR_INVALID;
    }
    const size_t off_words = 2 * ((size_t)num_envs + 1);
    const size_t off_words_al = (off_words + 63) & ~(size_t)63;  // keep the records 256-byte aligned
    const size_t need = off_words_al + (size_t)prm->max_contacts_per_body * num_bodies * kContactStride;
    if (need > kNoAllocWords) {
        set_error("vuda_sim_step_noalloc: batch needs " + std::to_string(need * 4) +
                  " bytes of scratch, more than the fixed " + std::to_string(kNoAllocWords * 4) +
                  " bytes (use vuda_env_create / vuda_sim_step, or a smaller batch)");
        return VUDA_ERR_INVALID;
    }
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess || dev < 0 || dev >= 64) {
        set_error(std::string("vuda_sim_step_noalloc: cudaGetDevice: ") + cudaGetErrorString(ce));
        return VUDA_ERR_CUDA;
    }
    void* base = nullptr;
    {
        ScratchAddr& sa = scratch_addr();
        std::lock_guard<std::mutex> lock(sa.mu);
        if (!sa.ptr[dev]) {
            // first call on this device: resolve the array's device address
            ce = cudaGetSymbolAddress(&sa.ptr[dev], g_noalloc_scratch);
            if (ce != cudaSuccess) {
                sa.ptr[dev] = nullptr;
                set_error(std::string("vuda_sim_step_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(ce));
                return VUDA_ERR_CUDA;
            }
        }
        base = sa.ptr[dev];
    }
    int64_t* spill_off = reinterpret_cast<int64_t*>(base);
    float* spill = reinterpret_cast<float*>(reinterpret_cast<uint32_t*>(base) + off_words_al);

    cudaStream_t s = (cudaStream_t)stream;
    spill_offsets_kernel<<<(num_envs + 1 + 255) / 256, 256, 0, s>>>(body_off, num_envs, prm->max_contacts_per_body,
                                                                     spill_off);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        set_error(std::string("vuda_sim_step_noalloc: offsets launch: ") + cudaGetErrorString(ce));
        return VUDA_ERR_CUDA;
    }
    DevBatch d{};
    d.E = num_envs;
    d.B = num_bodies;
    d.body_off = body_off;
    d.pos = pos;
    d.quat = quat;
    d.vel = vel;
    d.ang = angvel;
    d.type = shape_type;
    d.dims = shape_dims;
    d.im = inv_mass;
    d.ii = inv_inertia;
    d.pose[0] = pose;
    d.pose[1] = pose;
    d.flags = flags;
    d.ncontacts = ncontacts;
    d.spill = spill;
    d.spill_off = spill_off;
    SimConst k{};
    k.h = prm->dt / (float)prm->substeps;
    k.substeps = prm->substeps;
    k.iterations = prm->iterations;
    for (int i = 0; i < 3; i++) k.g[i] = prm->gravity[i];
    k.restitution = prm->restitution;
    k.rest_thr = prm->restitution_threshold;
    k.mu = prm->friction;
    k.beta = prm->baumgarte;
    k.slop = prm->slop;
    k.margin = prm->margin;
    k.omega = prm->jacobi_omega;
    k.plane = prm->plane;
    k.mcpb = prm->max_contacts_per_body;
    k.gyro = prm->gyroscopic;
    k.edges = prm->edge_contacts;
    k.hulls = 0;
    int smem = smem_per_env > 0 ? smem_per_env : phys_smem_bytes_default(max_bodies, k.mcpb);
    ce = launch_sim(d, k, nsteps, force, 0, smem, max_bodies, s);
    if (ce != cudaSuccess) {
        set_error(std::string("vuda_sim_step_noalloc: sim launch: ") + cudaGetErrorString(ce));
        return VUDA_ERR_CUDA;
    }
    return VUDA_OK;
}
