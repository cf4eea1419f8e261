// Internal declarations shared by the CUDA translation units of libvuda.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "vuda.h"

namespace vuda {

constexpr int kShapeSphere = 0;
constexpr int kShapeBox = 1;
constexpr int kShapeHull = 2;

struct SimConst {
    float h;                      // dt / substeps
    int substeps, iterations;
    float g[3];
    float restitution, rest_thr, mu, beta, slop, margin, omega;
    int plane, mcpb;
    int gyro;                     // gyroscopic term of boxes
    int edges;                    // box-box edge-edge contacts
    int hulls;                    // hull contacts from the hulls' vertices and faces
};

// Physics kernel variants: the code of an optional contact test is compiled
// only into the variants that carry its bit (a batch with the option off
// runs the variant without it).
constexpr int kFeatEdges = 1;
constexpr int kFeatHulls = 2;
__host__ __device__ inline int sim_features(const SimConst& k) {
    return (k.edges ? kFeatEdges : 0) | (k.hulls ? kFeatHulls : 0);
}

// Scratch of the tiled render path (tiled.cu), per camera c of env e with
// T_e triangles and n_c tiles (of the batch's tile size), R_e =
// tiled_record_cap(T_e) records (room for the extra fan triangles of
// near-plane clipping): records [rec_base, + R_e) of tiled_record_bytes()
// each, wide list [rec_base, + R_e), tile lists [ent_base, + bin_limit R_e),
// offsets [toff_base, + n_c + 2) (n_c + 1 list offsets, then the wide-list
// length).
struct TileScratch {
    void* rec;
    uint32_t* ent;
    uint32_t* wide;
    int32_t* toff;
};

// Device-resident batch.  All arrays are device pointers.
struct DevBatch {
    int E, B, C;
    const int32_t* body_off;      // [E+1]
    float* pos;                   // [3][B]
    float* quat;                  // [4][B]
    float* vel;                   // [3][B]
    float* ang;                   // [3][B]
    const uint8_t* type;          // [B]
    const float* dims;            // [3][B]
    const float* im;              // [B]
    const float* ii;              // [3][B]
    float* pose[2];               // [7][B] each: pos xyz, quat wxyz
    uint32_t* flags;              // [E]
    int32_t* ncontacts;           // [E] contacts at the last substep
    // physics contact spill area (contacts beyond the shared-memory capacity)
    float* spill;                 // [sum_e cmax_e * kContactStride] contact records that exceed shared memory
    const int64_t* spill_off;     // [E] first spill entry of env e (in contacts)
    // render
    const int32_t* mesh_id;       // [B]
    const float* scale;           // [3][B]
    const uint32_t* albedo;       // [B]
    const int32_t* mesh_vert_off; // [M+1]
    const float* mesh_verts;      // [V][3]
    const int32_t* mesh_tri_off;  // [M+1]
    const int32_t* mesh_tris;     // [T][3]
    const float4* mesh_plane;     // [T] face planes of the unit meshes: outward normal, offset (hull contacts)
    const float4* mesh_vert4;     // [V] the unit meshes' vertices padded to 16 bytes (hull contacts)
    int ground_mesh;
    uint32_t ground_albedo;
    const int32_t* cam_env;       // [C] env of camera c
    const int32_t* cam_w;
    const int32_t* cam_h;
    const float* cam_par;         // [C][13]: eye3 right3 up3 fwd3 fpy
    const int64_t* cam_pix_off;   // [C+1]
    const int64_t* env_tri_base;  // [E] first triangle of env e in the colour scratch
    uint32_t* tri_color;          // [sum_e tris_e] colour scratch
    const int64_t* body_tri_base; // [B] index in tri_color of body b's first triangle
    const int32_t* chunk_off;     // [E+1] render vertex-cache chunks of env e
    const int32_t* chunk_lo;      // [chunks] first env-local body of the chunk (-1 = ground quad)
    const int32_t* chunk_hi;      // [chunks] one past its last body
    const int32_t* chunk_tri0;    // [chunks] env-local id of the chunk's first triangle
    const int32_t* chunk_nv;      // [chunks] vertices of the chunk
    const int32_t* chunk_nt;      // [chunks] triangles of the chunk
    const int32_t* chunk_vtab;    // [chunks] first entry of the chunk's vertex table in vtab
    const int32_t* chunk_ttab;    // [chunks] first entry of the chunk's triangle table in ttab
    const int2* vtab;             // vertex v of a chunk: (mesh_verts index, body index k within the chunk)
    const uint2* ttab;            // triangle t of a chunk: chunk-local vertices (i0 | i1 << 16, i2)
    // vtab / ttab entries are shared by every chunk with the same sequence of meshes
    float light[3];
    SimConst sc;                  // physics constants of this batch
    vuda_frame frame;             // output frame (work-list launches; single-batch launches pass it)
    int max_bodies;               // largest environment of the batch
};

// Work-list items.  A launch either covers one batch directly (items == null:
// item i is environment i, or render work item i of the batch) or walks a
// list of items over several batches (descs[desc] for each item), pulled from
// an atomic counter by persistent CTAs.
//   sim item:    (desc | slot << 24, env)
//   render item: (desc | slot << 24, camera, first row, 0)
//   shade item:  (desc | slot << 24, unit)   unit < B: body, else ground of env unit - B
constexpr int kItemDescMask = 0xffffff;

// Per-SM admission of the CTAs of a work-list launch.  With SM-shared
// co-scheduling the sim and render launches each get a quota of CTAs per SM,
// so that both stay resident on every SM at once: a CTA stays only while
// fewer than `quota` CTAs of its launch hold a slot on its SM (slots[%smid]),
// otherwise it exits before taking work.  quota 0 admits every CTA.  The
// counts return to zero when the launch ends.
constexpr int kMaxSmSlots = 1024;
struct SmGate {
    int* slots;  // [kMaxSmSlots] device counters, zero between launches
    int quota;
};
constexpr int kGateOpen = -1;  // not gated (no quota, or an SM id beyond the table)
constexpr int kGateFull = -2;  // this SM already holds `quota` CTAs of the launch

#ifdef __CUDACC__
// Thread 0 of a CTA: take a slot on this SM.  Returns the SM id whose slot is
// held, kGateOpen, or kGateFull (the CTA must exit without work).
__device__ __forceinline__ int sm_gate_take(const SmGate& g) {
    if (g.quota <= 0 || g.slots == nullptr) return kGateOpen;
    unsigned sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    if (sm >= (unsigned)kMaxSmSlots) return kGateOpen;
    if (atomicAdd(g.slots + sm, 1) < g.quota) return (int)sm;
    atomicSub(g.slots + sm, 1);
    return kGateFull;
}
// Thread 0, once the CTA has finished: give back the slot it took (if any).
__device__ __forceinline__ void sm_gate_release(const SmGate& g, int held) {
    if (held >= 0) atomicSub(g.slots + held, 1);
}
#endif

// Resources one CTA of a work-list kernel holds on an SM.
struct CtaFootprint {
    int threads;
    int regs;   // per thread
    int smem;   // static + dynamic shared memory, bytes
};

constexpr int kContactWords = 32;  // floats per contact record: eight groups of four
// words between records: a multiple of four (16-byte groups) with an odd
// number of groups, so that 128-bit accesses by consecutive lanes to
// consecutive records fall in distinct bank groups
constexpr int kContactStride = kContactWords + 4;
constexpr int kCamWords = 13;

// Physics launchers (physics_impl.cuh): 128 threads per environment in
// namespace vuda (physics.cu), 512 in vuda::wide (physics_wide.cu).
#define VUDA_SIM_LAUNCHERS                                                                                      \
    cudaError_t launch_sim(const DevBatch& b, const SimConst& sc, int nsteps, const float* force,               \
                           int pose_slot_first, int smem_per_env, int max_bodies, cudaStream_t stream);         \
    /* Work-list form: grid CTAs pull items [0, nitems) from *counter (zeroed here on the stream first);     \
       max_bodies bounds every listed environment; force: optional [3][B] world forces, only for a list     \
       over one batch. */                                                                                     \
    cudaError_t launch_sim_items(const DevBatch* descs, const int2* items, int nitems, int* counter, int grid, \
                                 int smem_per_env, int max_bodies, const float* force, SmGate gate,           \
                                 int feat, cudaStream_t stream); /* feat: kFeat bits of any listed batch */     \
    int sim_ctas_per_sm(int smem_per_env);                                                                    \
    int sim_smem_for_ctas(int ctas); /* largest per-environment layout that keeps `ctas` CTAs per SM */        \
    CtaFootprint sim_list_footprint(int smem_per_env);                                                        \
    int phys_smem_bytes_default(int max_bodies, int mcpb);                                                    \
    int phys_min_smem_bytes(int max_bodies, int mcpb); /* the layout without contact records */               \
    int phys_contacts_in_smem(int smem_per_env, int max_bodies, int mcpb);
VUDA_SIM_LAUNCHERS
namespace wide {
VUDA_SIM_LAUNCHERS
}
constexpr int kWideBodies = 64;   // environments with more bodies take the 512-thread physics kernel
// Launchers (render.cu, tiled.cu)
cudaError_t launch_render_items(const DevBatch& b, const float* pose, const vuda_frame& fr, const int32_t* item_cam,
                                const int32_t* item_y0, int nitems, int band_rows, int max_w, cudaStream_t stream);
// Work-list form over several batches (frames from each descriptor).
cudaError_t launch_render_list(const DevBatch* descs, const int4* items, int nitems, int* counter, int grid,
                               const int2* shade_items, int nshade, int band_rows, int max_w, const vuda_frame* fr0,
                               SmGate gate, cudaStream_t stream);
int render_ctas_per_sm(int band_rows, int max_w);
CtaFootprint render_list_footprint(int band_rows, int max_w);
size_t render_smem_for(int band_rows, int W);
int render_default_band_rows(int max_w, int max_h);
int render_chunk_bodies();
cudaError_t launch_raster_screen(const int32_t* xy, const float* z, int ntri, int W, int H, uint32_t* triid,
                                 float* depth, uint32_t* count, cudaStream_t stream);
int render_vcap();
// Per-triangle flat colours of the batch for the poses `pose` (render.cu).
cudaError_t launch_shade(const DevBatch& b, const float* pose, cudaStream_t stream);

// A camera (bin_kernel, tile0 = 0) or a raster work item of
// tiled_tiles_per_item() tiles from tile0 (tile_kernel), with everything the
// kernels need about the camera in one 80-byte record.
struct __align__(16) TileItem {
    int cam, tile0, W, H;         // bytes 0..15
    int tiles_x, ntiles, env, pad;  // 16..31
    long long rec_base, ent_base; // 32..47
    long long toff_base, rec_cap; // 48..63: rec_cap = records (and wide-list entries) of the camera
    long long pix_off;            // 64: first pixel of the camera in the frame
    long long col_base;           // 72: first triangle of the environment in the colour table
};
int tiled_max_tiles();               // tiles per camera the path supports
int tiled_default_bin_limit();       // list entries per triangle at most, by default
int tiled_max_bin_limit();
int tiled_tiles_per_item(int tile);  // tiles per raster work item for tile size 8, 16 or 32
size_t tiled_record_bytes();
// Record slots of a camera whose environment has T triangles: T, plus an
// eighth for the second fan triangle of a triangle clipped to a
// quadrilateral at the near plane (bin_kernel flags VUDA_FLAG_CLIP_CAPACITY
// and drops what does not fit).
inline long long tiled_record_cap(long long T) { return T + T / 8 + 8; }
// Set up, shade and bin every camera into tile x tile tiles (8, 16, 32),
// listing a triangle under at most nlim tiles (else on the wide list), then
// rasterise and resolve the work items (camera, first tile) of
// tiled_tiles_per_item(tile) tiles each.
// Face planes of every triangle of the mesh library (hull contacts): for
// triangle t of mesh m with unit-mesh vertices u0, u1, u2, c = (u1 - u0) x
// (u2 - u0), the outward unit normal n = c / |c| and the offset n . u0
// (planes[t] = (n, offset)); a triangle of zero area gets (0, 0, 0, +inf).
cudaError_t launch_mesh_planes(const float* verts, const int32_t* vert_off, const int32_t* tri_off,
                               const int32_t* tris, int num_meshes, int num_tris, float4* planes, int num_verts,
                               float4* vert4, cudaStream_t stream);

// Pooled observation of frame fr (vuda_observe): every camera's cells x
// cells cells (camera sizes divisible by cells), mean depth x depth_scale and
// mean luminance, into out[E][2 cams_per_env cells^2].
cudaError_t launch_observe(const DevBatch& b, const vuda_frame& fr, int cams_per_env, int cells, float depth_scale,
                           float* out, cudaStream_t stream);

// sieve: set-up in two passes (keep the triangles that can leave a record,
// then set them up with full warps), for batches whose triangles outnumber
// their pixels
cudaError_t launch_render_tiled(const DevBatch& b, const float* pose, const vuda_frame& fr, const TileScratch& ts,
                                const TileItem* cams, const TileItem* items, int nitems, int tile, int nlim, bool sieve,
                                cudaStream_t stream);
// One batch of a tiled work list over several batches: its device camera
// and raster items and its scratch (as built for its own launches), the
// list positions of its first camera and first raster item, and
// `desc | slot << 24`.  (The scratch is kept here, not in DevBatch: the
// physics kernels copy DevBatch into shared memory, where 7 CTAs per SM
// leave no room for it to grow.)
struct TiledJob {
    const TileItem* cams;
    const TileItem* items;
    TileScratch ts;
    int cam0, item0;
    int tag;
    int pad;
};
// Work-list form over several batches with the default tile size and bin
// limit: camera k of the list is camera k - cam0 of the job holding it (the
// last job with cam0 <= k), likewise for raster items; batch descs[desc]
// renders from its pose slot into its own frame (DevBatch::frame) with the
// job's tiled scratch.
cudaError_t launch_render_tiled_list(const DevBatch* descs, const TiledJob* jobs, int njobs, int ncams, int nitems,
                                     cudaStream_t stream);
int tiled_default_tile();
// Tiled scratch bytes of a scene at the default tile size and bin limit
// (0 if a camera has more tiles than the path supports).
int64_t tiled_scratch_estimate(const vuda_scene* sc);

void set_error(const std::string& s);
// Device bytes a batch will hold once created (an upper estimate).
vuda_status env_estimate_bytes(const vuda_scene* sc, const vuda_sim_params* p, int64_t* out);

}  // namespace vuda
