// The environment-batch handle shared by the C-ABI translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "internal.cuh"

struct vuda_env {
    int device = 0;
    vuda::DevBatch d{};
    vuda::SimConst sc{};
    vuda_sim_params params{};
    int E = 0, B = 0, C = 0, max_bodies = 0, max_w = 0;
    int64_t P = 0, T = 0;
    int64_t bytes = 0;
    int64_t steps = 0;
    int phys_smem = 0;
    int phys_smem_user = 0;        // the caller's shared memory per env (0: automatic)
    int band_rows = 0;
    int nitems = 0;
    int32_t* item_cam = nullptr;
    int32_t* item_y0 = nullptr;
    std::vector<void*> allocs;
    std::vector<int64_t> cam_pix_off;
    std::vector<int32_t> h_item_cam, h_item_y0;   // host copies of the render work items
    std::vector<int32_t> h_cam_w, h_cam_h, h_cam_env, h_body_off;
    std::vector<int64_t> h_env_tri_base;
    int max_h = 0;
    // co-scheduling
    int cos_mode = 0;
    cudaStream_t sim_s = nullptr, ren_s = nullptr;
    cudaStream_t own_s = nullptr;                 // primary-context stream of the rollout policy beside green partitions
    CUgreenCtx g_sim = nullptr, g_ren = nullptr;
    CUcontext c_sim = nullptr, c_ren = nullptr;  // green contexts as CUcontext (null otherwise)
    vuda_cosched_info cos_info{};
    std::vector<cudaEvent_t> ev_sim, ev_ren;      // event pools owned by each phase's context
    // persistent work-list launches (uneven batches)
    int persistent = 0;
    vuda::DevBatch* d_desc = nullptr;                   // device copy of d
    int2* sim_items[2] = {nullptr, nullptr};      // per pose slot: (0 | slot << 24, env), largest first
    // the same environments by size class for the persistent physics: each
    // class has its own shared-memory layout (its largest environment), CTA
    // size and work list
    struct SimClass {
        int2* items[2] = {nullptr, nullptr};
        int nitems = 0, max_bodies = 0, smem = 0, grid = 0, wide = 0;
    };
    std::vector<SimClass> sim_classes;
    // the size classes after the first run on streams of their own, forked
    // from and joined back into the sim stream (independent environments)
    std::vector<cudaStream_t> class_s;
    std::vector<cudaEvent_t> class_join;
    cudaEvent_t class_fork = nullptr;
    int class_prio = 0;
    int4* ren_items[2] = {nullptr, nullptr};      // per pose slot: (0 | slot << 24, cam, y0, 0), largest first
    int2* shade_items[2] = {nullptr, nullptr};
    int nshade = 0;
    int* counters = nullptr;                      // [2 + size classes]: sim, render, one per physics class
    int sim_grid = 0, ren_grid = 0;
    int lists = 0;                                // the work lists above are built
    // SM-shared co-scheduling: per-SM slot counters ([2][kMaxSmSlots]: sim,
    // render), CTAs per SM of each phase and the launch grids
    int* sm_slots = nullptr;
    int sim_quota = 0, ren_quota = 0;
    int sim_grid_sh = 0, ren_grid_sh = 0;
    // tiled render path: scratch and work items (camera, first tile)
    int tiled = 0;
    int tile_size = 16, bin_limit = 9;   // tile edge in pixels; most tile lists a triangle joins
    int64_t tiled_nent = 0, tiled_ntoff = 0;   // elements of ts.ent and ts.toff
    vuda::TileScratch ts{};
    vuda::TileItem* tcams = nullptr;    // [C]
    vuda::TileItem* titems = nullptr;   // [ntitems]
    int ntitems = 0;
    // captured pipeline (CUDA graph of gsteps pipelined steps)
    cudaGraphExec_t gexec = nullptr;
    int gsteps = 0, gparity = 0, gmode = 0;
    vuda_frame gring[2] = {};
    // host-buffer loop: device force ring and a copy stream (primary context)
    float* dforce = nullptr;                      // [2][3][B]
    cudaStream_t copy_s = nullptr;
    cudaEvent_t copy_done[2] = {nullptr, nullptr};
};
