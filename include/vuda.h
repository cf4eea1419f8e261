/* vuda.h -- C ABI of the co-scheduled simulate-then-render library (libvuda.so).
 *
 * The paper (VUDA, arxiv 2605.01352) speeds up the per-step loop of
 * embodied-AI environments -- a physics step followed by a camera render --
 * by letting the two phases share the GPU spatially instead of in alternating
 * time slices.  Its application interface (Sec. 3.2, Table 1) binds a stream
 * for co-scheduling (CUstream_bind / CUstream_unbind) and launches the two
 * phases asynchronously (step_async / render_async) with blocking waits
 * (wait_step / wait_render).  Sec. 3.1 gives the dependency this exploits:
 * sim(k+1) depends only on sim(k), never on render(k).
 *
 * This library computes both phases itself in CUDA (sm_103a) in one context:
 * a batched rigid-body step and a batched per-environment rasteriser, with
 * the sim and render streams placed on disjoint SM partitions.
 *
 * Conventions for every entry point:
 *  - Nothing aborts or throws across the ABI; every call returns a
 *    vuda_status.  VUDA_ERR_CUDA carries the CUDA error text, available from
 *    vuda_last_error().
 *  - Host input pointers are read only during the call.  Device pointers
 *    given by the caller (frames, forces) stay owned by the caller; the
 *    library never frees caller memory.  The library owns all device memory
 *    it allocates for an environment batch and frees it in vuda_env_destroy.
 *  - Streams are cudaStream_t values passed as void*; NULL is the legacy
 *    default stream.  Calls named *_step / *_render only enqueue work.
 *  - Arrays called SoA are planes: pos[3][B] is x[0..B), y[0..B), z[0..B).
 *  - A handle may be used from one host thread at a time.
 */
#ifndef VUDA_H
#define VUDA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VUDA_OK = 0,
    VUDA_ERR_INVALID = 1,      /* bad argument or size */
    VUDA_ERR_OOM = 2,          /* device allocation failed or HBM budget exceeded */
    VUDA_ERR_CUDA = 3,         /* a CUDA call failed; see vuda_last_error() */
    VUDA_ERR_OVERFLOW = 4,     /* a capacity was exceeded (see the env flags) */
    VUDA_ERR_TIMEOUT = 5,      /* a bounded wait gave up (vuda_serve_poll with wait_ms > 0) */
    VUDA_ERR_BUSY = 6,         /* resource in use (e.g. serving queue full) */
    VUDA_ERR_UNSUPPORTED = 7   /* feature not available on this device/driver */
} vuda_status;

/* Per-environment status bits (vuda_env_status).  They accumulate until
 * cleared and never stop the step: the work degrades deterministically. */
#define VUDA_FLAG_CONTACT_OVERFLOW 0x1u /* contacts beyond max_contacts_per_body * N dropped */
#define VUDA_FLAG_CLIP_CAPACITY    0x2u /* tiled path: a triangle found no record slot (only the extra fan
                                            triangles of near-plane clipping can need more slots than the
                                            camera has triangles) and was skipped */
#define VUDA_FLAG_GUARD_DISCARD    0x4u /* a triangle beyond the 2^14 px guard band was skipped */
#define VUDA_FLAG_MESH_CAPACITY    0x8u /* a mesh larger than the render vertex cache was skipped */
#define VUDA_FLAG_BAD_RANGE        0x10u /* the environment's body range was invalid (outside the batch, or more
                                            bodies than max_bodies): the environment was skipped, nothing written */

typedef void* vuda_stream_t;        /* cudaStream_t */
typedef struct vuda_env* vuda_env_t;

/* Physics step parameters.  A step of length dt is split into `substeps`
 * substeps of h = dt / substeps; each substep integrates velocities, builds
 * contacts, runs `iterations` Jacobi iterations and integrates positions. */
typedef struct {
    float dt;
    int32_t substeps;
    int32_t iterations;
    float gravity[3];
    float restitution;            /* applied to penetrating contacts approaching faster than the threshold */
    float restitution_threshold;
    float friction;               /* Coulomb coefficient (disk cone) */
    float baumgarte;              /* position bias factor beyond the slop */
    float slop;                   /* allowed penetration (m) */
    float margin;                 /* speculative contact distance (m) */
    float jacobi_omega;           /* relaxation of the mass-split Jacobi update */
    int32_t plane;                /* 1: static ground plane z = 0 */
    int32_t max_contacts_per_body;/* contact capacity per env = this * bodies */
    int32_t gyroscopic;           /* 1: gyroscopic term of boxes, I dw/dt = -w x I w in the body frame, one
                                     implicit (Newton) step per substep; spheres and hull proxies have none */
    int32_t edge_contacts;        /* 1: box-box edge-edge contacts (separating-axis test over 15 axes; one
                                     contact between crossing edges, after the pair's corner contacts) */
    int32_t hull_contacts;        /* 1: hulls collide as the convex hulls of their meshes scaled by dims[0]
                                     (their vertices on the plane; a sphere's centre against the deepest face;
                                     hull-hull and hull-box: separating-axis test over the face normals, the
                                     incident face clipped by the reference face's sides), after all other
                                     contacts; 0: hulls are spheres of radius dims[0].  Not accepted by
                                     vuda_sim_step_noalloc (no meshes there) */
} vuda_sim_params;

/* Host description of a batch (all arrays host memory, read during
 * vuda_env_create only).  E environments, B = body_off[E] bodies,
 * C = cam_off[E] cameras, M meshes.
 *   body_off[E+1]           CSR: env e owns bodies [body_off[e], body_off[e+1])
 *   pos[3][B] quat[4][B]    pose (quat = w, x, y, z, unit)
 *   vel[3][B] angvel[3][B]  linear / angular velocity (world frame)
 *   shape_type[B]           0 sphere, 1 box, 2 hull (a sphere of radius dims[0] unless hull_contacts)
 *   shape_dims[3][B]        sphere/hull: (r, -, -); box: half extents
 *   inv_mass[B] inv_inertia[3][B]   body-frame principal inverse inertia
 *   mesh_id[B] mesh_scale[3][B] albedo[B] (r | g<<8 | b<<16)
 *   mesh_vert_off[M+1] mesh_verts[V][3]  mesh_tri_off[M+1] mesh_tris[T][3] (mesh-local,
 *                           counter-clockwise seen from outside)
 *   ground_mesh             mesh drawn once per env in world coordinates (ids 0..)
 *   cam_off[E+1] cam_w[C] cam_h[C] cam_eye/right/up/fwd[C][3] cam_fpy[C]  pinhole cameras
 *   light[3]                unit direction towards the light */
typedef struct {
    int32_t num_envs;
    const int32_t* body_off;
    const float* pos;
    const float* quat;
    const float* vel;
    const float* angvel;
    const uint8_t* shape_type;
    const float* shape_dims;
    const float* inv_mass;
    const float* inv_inertia;
    const int32_t* mesh_id;
    const float* mesh_scale;
    const uint32_t* albedo;
    int32_t num_meshes;
    const int32_t* mesh_vert_off;
    const float* mesh_verts;
    const int32_t* mesh_tri_off;
    const int32_t* mesh_tris;
    int32_t ground_mesh;
    uint32_t ground_albedo;
    const int32_t* cam_off;
    const int32_t* cam_w;
    const int32_t* cam_h;
    const float* cam_eye;
    const float* cam_right;
    const float* cam_up;
    const float* cam_fwd;
    const float* cam_fpy;
    float light[3];
} vuda_scene;

/* Creation options.  Zero-initialised options are valid (defaults). */
typedef struct {
    int64_t hbm_budget_bytes;     /* 0: no limit; else VUDA_ERR_OOM if the batch needs more */
    int32_t device;               /* CUDA device ordinal (default 0) */
    int32_t render_band_rows;     /* rows per render work item (0: auto) */
    int32_t phys_smem_bytes;      /* shared memory per physics env (0: auto) */
    int32_t persistent;           /* 1: one persistent launch per phase pulls work items (environments,
                                     camera bands) largest first from an atomic counter -- for batches of
                                     uneven environments; 0: one CTA per item */
    int32_t render_path;          /* VUDA_RENDER_AUTO / _BAND / _TILED (see below) */
    int32_t tile_size;            /* tiled path: tile edge, 8, 16 or 32 pixels (0: 16) */
    int32_t tile_bin_limit;       /* tiled path: most tile lists one triangle joins; triangles over more
                                     tiles go to the camera's wide list, read by every tile (1..64, 0: 9) */
} vuda_env_opts;

/* Render paths (identical frames; they differ in how work is split):
 * BAND: one CTA per band of rows of a camera sets up every triangle of the
 * environment and rasterises the band in shared memory.  TILED: one CTA per
 * camera sets up every triangle once into a device scratch area and bins it
 * into tile_size x tile_size tiles, then one warp per tile rasterises and
 * resolves it (needs cameras of at most 2048 tiles, e.g. 640 x 480 at 16 x 16,
 * and scratch of about 84 + 4 tile_bin_limit bytes per triangle and camera, an
 * upper bound of which only the visible part is written).  AUTO: TILED where it applies and its scratch
 * fits (at most half of the free device memory, and within
 * hbm_budget_bytes), else BAND.
 * The render work-list launches of VUDA_COSCHED_SHARED use the band kernel;
 * the serving loop renders each job on the path its batch chose (work lists
 * over several jobs for both); persistent = 1 makes the physics a work-list
 * launch and keeps the chosen render path. */
#define VUDA_RENDER_AUTO 0
#define VUDA_RENDER_BAND 1
#define VUDA_RENDER_TILED 2

/* Sizes of a created batch. */
typedef struct {
    int32_t num_envs, num_bodies, num_cams, max_bodies;
    int64_t num_pixels;           /* total pixels over all cameras */
    int64_t num_tris;             /* total triangles drawn per step over all envs (per camera) */
    int64_t device_bytes;         /* device memory held by the batch */
    int64_t steps_enqueued;       /* physics steps enqueued so far */
    int32_t render_path;          /* VUDA_RENDER_BAND or VUDA_RENDER_TILED: the path the batch renders with */
    int32_t tile_size, tile_bin_limit;   /* the tiled path's raster parameters (0 on the band path) */
} vuda_env_info;

/* Caller-owned device output buffers, concatenated per camera in cam order
 * (pixel p of camera c at cam_pix_off[c] + y * W + x):
 *   rgb[P][3] u8, depth[P] f32 (view depth, 0 = background),
 *   triid[P] u32 (env-local triangle id, 0xFFFFFFFF = background; may be NULL). */
typedef struct {
    uint8_t* rgb;
    float* depth;
    uint32_t* triid;
} vuda_frame;

/* Host state (SoA planes of length B); used by get/set. */
typedef struct {
    float* pos;
    float* quat;
    float* vel;
    float* angvel;
} vuda_state;

const char* vuda_status_str(vuda_status s);
/* Text of the last error raised on this thread (empty if none). */
const char* vuda_last_error(void);
int32_t vuda_abi_version(void);

/* Create a batch: validates the description (VUDA_ERR_INVALID), checks the
 * HBM budget (VUDA_ERR_OOM), uploads state, meshes and cameras.  Synchronous.
 * Problem statement: Sec. 3.1 (a batch of environments stepped and rendered
 * in a loop). */
vuda_status vuda_env_create(const vuda_scene* scene, const vuda_sim_params* params,
                            const vuda_env_opts* opts, vuda_env_t* out);
vuda_status vuda_env_destroy(vuda_env_t env);
/* Device bytes vuda_env_create would hold for this batch (an upper estimate,
 * the figure the serving loop admits jobs by).  Host only. */
vuda_status vuda_env_estimate_bytes(const vuda_scene* scene, const vuda_sim_params* params, int64_t* bytes);
vuda_status vuda_env_info_get(vuda_env_t env, vuda_env_info* out);
/* Per-camera first-pixel offsets (host array of num_cams + 1). */
vuda_status vuda_env_cam_pix_off(vuda_env_t env, int64_t* out);

/* Enqueue nsteps physics steps on `stream` (the paper's step_async, Table 1).
 * force: optional device array [3][B] of world forces held over each step
 * (NULL: none).  After each step the body poses are also written to pose
 * slot (step index mod 2) for the renderer.  Async; returns after enqueue. */
vuda_status vuda_sim_step(vuda_env_t env, int32_t nsteps, const float* force, vuda_stream_t stream);

/* Enqueue the render of every camera from pose slot `pose_slot` (0 or 1;
 * -1 = the slot of the last enqueued step) into `frame` (the paper's
 * render_async, Table 1).  Async. */
vuda_status vuda_render(vuda_env_t env, int32_t pose_slot, const vuda_frame* frame, vuda_stream_t stream);

/* Co-scheduling (the paper's CUstream_bind, Table 1 / Sec. 3.2):
 * mode VUDA_COSCHED_GREEN puts a sim stream and a render stream on disjoint
 * SM partitions (green contexts, sim_sms SMs for sim, the rest for render);
 * VUDA_COSCHED_STREAMS uses two ordinary streams that share all SMs;
 * VUDA_COSCHED_SHARED partitions every SM instead of the set of SMs: both
 * phases run as persistent work-list launches, and a CTA is admitted only
 * while its SM holds fewer than sim_ctas_per_sm (render_ctas_per_sm) CTAs of
 * its phase, so that sim(t+1) and render(t) are resident side by side on
 * every SM (0: a default pair that fits; VUDA_ERR_INVALID if a pair does not
 * fit one SM together).
 * The streams are owned by the library and returned for the caller to
 * enqueue on.  vuda_coschedule_reset (CUstream_unbind) destroys them. */
#define VUDA_COSCHED_STREAMS 1
#define VUDA_COSCHED_GREEN 2
#define VUDA_COSCHED_SHARED 3
typedef struct {
    int32_t mode;
    int32_t sim_sms;              /* GREEN: SMs for the sim partition (0: half); rounded to the device granularity */
    int32_t sim_ctas_per_sm;      /* SHARED: sim CTAs per SM (0: default) */
    int32_t render_ctas_per_sm;   /* SHARED: render CTAs per SM (0: default) */
    int32_t priority;             /* VUDA_PRIORITY_*: which stream's CTAs the block scheduler dispatches first
                                     when both have work (STREAMS and SHARED share SMs) */
} vuda_cosched_opts;
#define VUDA_PRIORITY_NONE 0
#define VUDA_PRIORITY_SIM 1
#define VUDA_PRIORITY_RENDER 2
typedef struct {
    int32_t mode;
    int32_t sim_sms, render_sms;  /* SMs actually provisioned (0 if not partitioned) */
    int32_t sm_granularity;       /* partition alignment reported by the driver */
    int32_t sim_ctas_per_sm, render_ctas_per_sm;  /* SHARED: the per-SM quotas in use */
    int32_t priority;
} vuda_cosched_info;
vuda_status vuda_coschedule(vuda_env_t env, const vuda_cosched_opts* opts, vuda_stream_t* sim_stream,
                            vuda_stream_t* render_stream, vuda_cosched_info* info);
vuda_status vuda_coschedule_reset(vuda_env_t env);

/* Optional timing of a loop run (host arrays of nsteps entries, each may be
 * NULL), from device events:
 *   step_ms[t]   start of sim(t) to the end of render(t) (step latency)
 *   sim_ms[t]    duration of sim(t) on the sim stream
 *   render_ms[t] duration of render(t) on the render stream
 *   total_ms     start of sim(0) to the end of render(nsteps-1)
 * Intervals between the two co-scheduled streams are NaN if the driver
 * cannot relate their events. */
typedef struct {
    float* step_ms;
    float* sim_ms;
    float* render_ms;
    float total_ms;
} vuda_timing;

/* Run nsteps steps of the loop and block until done.  Co-scheduled
 * (after vuda_coschedule): sim(t+1) is enqueued on the sim stream as soon as
 * sim(t) is, render(t) on the render stream after sim(t) (Sec. 3.1 inter-step
 * pipelining); frames alternate between ring[0] and ring[1] and pose slots
 * alternate too, guarded by events.  Not co-scheduled: sim then render on
 * `stream`.  timing may be NULL. */
vuda_status vuda_pipeline_run(vuda_env_t env, int32_t nsteps, const vuda_frame* ring, vuda_stream_t stream,
                              vuda_timing* timing);

/* Capture steps_per_graph (even) pipelined steps of the loop -- as
 * vuda_pipeline_run would enqueue them with this ring and the current
 * co-scheduling -- into a CUDA graph.  Later vuda_pipeline_run calls with the
 * same ring, a multiple of steps_per_graph steps and the same pose-slot
 * parity replay the graph instead of launching kernel by kernel (step
 * latencies are then reported as NaN).  Returns VUDA_ERR_UNSUPPORTED if the
 * driver refuses the capture.  Invalidated by vuda_coschedule*. */
vuda_status vuda_pipeline_capture(vuda_env_t env, int32_t steps_per_graph, const vuda_frame* ring,
                                  vuda_stream_t stream);
vuda_status vuda_pipeline_release_graph(vuda_env_t env);

/* Batching layer, raster parameters (the paper's renderer is Vulkan's and has
 * no such knobs; these are what the autotuner below chooses between).
 * Raster parameters of a batch on the tiled render path: tile edge (8, 16 or
 * 32 pixels) and bin limit (1..64; see vuda_env_opts).  Reallocates the
 * path's tile lists (VUDA_ERR_INVALID on the band path, for cameras of more
 * than 2048 tiles, or when the lists would exceed half of the free device
 * memory; the batch keeps its previous parameters then).  Frames do not
 * depend on the choice.  Drops a captured graph.  Synchronous. */
vuda_status vuda_set_tiling(vuda_env_t env, int32_t tile_size, int32_t bin_limit);

/* Autotuner: measures the loop under candidate configurations -- render band
 * height (16/32/64/128 rows) on the band path, or tile size (8/16/32) x bin
 * limit (4/9/16) on the tiled path, serialized / co-scheduled on shared SMs /
 * co-scheduled on disjoint partitions of 1/4, 1/2 and 3/4 of the SMs /
 * co-scheduled with per-SM quotas (every pair that fits one SM, the most sim
 * CTAs for each render count), and CUDA graph replay -- and leaves the batch
 * configured with the fastest; co-scheduling and graph replay are kept only
 * when they beat the configuration before them by more than 1 % (the
 * trials' noise).  Results are cached per batch shape for the process
 * (use_cache = 1 reuses them without measuring).  Every trial starts from
 * the batch's state at the call; the state and pose slots are restored
 * afterwards.  ring: the two frames the loop will use. */
typedef struct {
    int32_t steps;                /* measured steps per trial (0: 6) */
    int32_t use_cache;
} vuda_tune_opts;
typedef struct {
    int32_t band_rows, cosched_mode, sim_sms, graph_steps;
    float ms_per_step, ms_per_step_serialized;
    int32_t trials, from_cache;
    int32_t sim_ctas_per_sm, render_ctas_per_sm;  /* SHARED winner's quotas */
    int32_t priority;                             /* the winner's stream priority */
    int32_t tile_size, tile_bin_limit;            /* tiled path: the chosen raster parameters (0: band path) */
} vuda_tune_result;
vuda_status vuda_autotune(vuda_env_t env, const vuda_tune_opts* opts, const vuda_frame* ring, vuda_tune_result* out);

/* The same loop with host buffers (end-to-end use): each step copies its
 * force input from host memory (h_force: [3][B] floats, or [nsteps][3][B]
 * when force_per_step != 0; NULL for none) to the device before sim(t), and
 * copies the frame of step t (RGB and depth) from the device ring slot t & 1
 * into the host ring slot t & 1 (h_rgb: [2][P][3] bytes, h_depth: [2][P]
 * floats) on a copy stream, overlapped with the following steps.  Host
 * buffers must be page-locked for the copies to be asynchronous.  ring: the
 * two device frames used as staging.  Blocks until everything is done. */
vuda_status vuda_pipeline_run_host(vuda_env_t env, int32_t nsteps, const float* h_force, int32_t force_per_step,
                                   uint8_t* h_rgb, float* h_depth, const vuda_frame* ring, vuda_stream_t stream,
                                   vuda_timing* timing);

/* RL rollout with the inter-trajectory schedule (Sec. 3.1, RL training:
 * within a trajectory inference(k+1) depends on render(k), but different
 * trajectories are independent; Sec. 6.4 runs the policy, physics and
 * rendering on one GPU).  The trajectories form two groups, each its own
 * batch (g0, g1), and each step of a group is sim -> render -> policy: the
 * sim uses the group's forces (device [3][B_g], force0 / force1), the
 * render writes frame ring_g[k & 1] from the new poses, and the policy reads
 * that frame and writes the forces of the group's next step.  The policy is
 * the caller's: `policy` is called on this thread, in step order, to
 * ENQUEUE its work on the stream it is given (it must not synchronise);
 * `step` is the group's step just rendered; a nonzero return aborts the
 * run (VUDA_ERR_INVALID).  The first step uses the forces the arrays hold.
 * Schedule: co-scheduled (vuda_coschedule on g0 with VUDA_COSCHED_STREAMS or
 * _GREEN; g1 must not be co-scheduled: it uses g0's streams), one group's
 * sim runs on the sim stream while the other group's render and policy run
 * on the render stream:
 *   sim stream:     sim(0,k) sim(1,k)        sim(0,k+1)         sim(1,k+1) ...
 *   render stream:           ren(0,k) pol(0,k) ren(1,k) pol(1,k) ren(0,k+1) ...
 * (with GREEN partitions the policy runs on a primary-context stream of its
 * own, ordered by events).  Not co-scheduled: the same order on `stream`,
 * one phase at a time (time slicing).  Results do not depend on the
 * schedule.  timing (may be NULL): total_ms from the first sim to the last
 * policy (NaN if the driver cannot relate the events).  Blocks until done. */
typedef int32_t (*vuda_policy_fn)(void* user, int32_t group, int64_t step, const vuda_frame* frame, float* force,
                                  vuda_stream_t stream);
vuda_status vuda_rollout_run(vuda_env_t g0, vuda_env_t g1, int32_t nsteps, const vuda_frame* ring0,
                             const vuda_frame* ring1, float* force0, float* force1, vuda_policy_fn policy,
                             void* user, vuda_stream_t stream, vuda_timing* timing);

/* Pooled observation of a rendered frame, for a policy acting between steps
 * (the action generator of the RL rollout reads it; the paper has no
 * counterpart: its policies read the Vulkan images).  Each camera's image is
 * cut into cells x cells equal cells; a cell gives its mean view depth times
 * depth_scale and its mean luminance (0.299 r + 0.587 g + 0.114 b) / 255,
 * each summed over the cell's pixels row by row.  out (device, E x 2 C_e
 * cells^2 floats, C_e the cameras per environment) holds per environment
 * the depth means of its cameras in order (cells row-major), then the
 * luminance means in the same order.  Every environment must have the same
 * number of cameras and every camera a width and height divisible by cells
 * (1 <= cells <= 64), and frame its rgb and depth buffers, else
 * VUDA_ERR_INVALID.  Async on stream (capturable). */
vuda_status vuda_observe(vuda_env_t env, const vuda_frame* frame, int32_t cells, float depth_scale, float* out,
                         vuda_stream_t stream);

/* Block until all work enqueued by this handle on the sim (phase 0) or
 * render (phase 1) stream has finished (wait_step / wait_render, Table 1). */
vuda_status vuda_wait(vuda_env_t env, int32_t phase);

/* Copy the state to / from host SoA arrays (synchronous).  Not in the paper
 * (its loop never leaves the device): checkpoint / resume of a batch, and
 * the common starting state of parity checks. */
vuda_status vuda_env_get_state(vuda_env_t env, const vuda_state* out);
vuda_status vuda_env_set_state(vuda_env_t env, const vuda_state* in);
/* Read the pose slot (pos[3][B], quat[4][B]) to host.  Not in the paper: the
 * renderer reads pose slots in place (the zero-copy sharing of Sec. 3.1);
 * these copies serve inspection and rendering of given poses. */
vuda_status vuda_env_get_pose(vuda_env_t env, int32_t slot, float* pos, float* quat);
/* Write a pose slot from host arrays (used to render given poses). */
vuda_status vuda_env_set_pose(vuda_env_t env, int32_t slot, const float* pos, const float* quat);

/* Read (and optionally clear) per-env status bits into flags[E] (host, may
 * be NULL); or_flags receives their union.  Synchronous.  Not in the paper:
 * the kernels' record of deterministic degradation (VUDA_FLAG_*). */
vuda_status vuda_env_status(vuda_env_t env, uint32_t* flags, uint32_t* or_flags, int32_t clear);
/* Number of contacts of each env at the last substep (host int32[E]).  Not
 * in the paper: a diagnostic of the collision stage of Sec. 2.1. */
vuda_status vuda_env_contact_counts(vuda_env_t env, int32_t* counts);

/* Test entry point: rasterise ntri screen-space triangles with snapped 24.8
 * fixed-point vertices xy[t][3][2] (int32) and view depths z[t][3] into a
 * W x H image (all device pointers): triid[H][W] u32 (0xFFFFFFFF empty),
 * depth[H][W] f32 (0 empty), count[H][W] u32 (may be NULL: number of
 * triangles covering each pixel).  Same coverage rule and depth key as
 * vuda_render; triangle ids are the input order.  As in vuda_render, a
 * triangle with a vertex beyond the 2^14-pixel guard band (|x| or |y| above
 * 2^22) is discarded.  Async on `stream`. */
vuda_status vuda_raster_screen_tris(const int32_t* xy, const float* z, int32_t ntri, int32_t W, int32_t H,
                                    uint32_t* triid, float* depth, uint32_t* count, vuda_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of step+render requests from many jobs.     */
/* ------------------------------------------------------------------------ */
/* Not in the paper, which runs one data-generation or rollout job at a time
 * (Sec. 6.3, 6.4); this is the request loop that serves many such jobs at
 * once on one GPU.
 * A job is a batch of environments (a vuda_scene plus sim params) that stays
 * resident on the device once admitted.  A request asks for one physics step
 * of all the job's environments followed by the render of all its cameras.
 * Jobs are admitted in arrival order while their device memory fits
 * hbm_budget_bytes (0: no limit); a worker thread batches the pending
 * request of every admitted job into one launch per phase, and pipelines the
 * launches (the sim phase of the next batch overlaps the render phase of the
 * current one), so requests arriving while others run join the next batch.
 * A job's results are the same alone and in any mix.
 * Host-side fault injection (read when the server is created; no GPU fault
 * is made): VUDA_FAULT_REJECT_JOB=<job id> refuses that job's admission (its
 * requests complete with VUDA_ERR_INVALID); VUDA_FAULT_OOM_JOB=<job id>
 * fails its admission as if its device memory could not be allocated
 * (VUDA_ERR_OOM); VUDA_FAULT_STALL_MS=<ms> and VUDA_FAULT_STALL_EVERY=<n>
 * stall the batching worker for ms before every n-th launch.  Job ids count
 * from 1 in the order jobs are added. */
typedef struct vuda_server* vuda_server_t;
typedef struct {
    int32_t device;
    int64_t hbm_budget_bytes;     /* admission limit for resident jobs (0: none) */
    int32_t max_jobs;             /* resident jobs at once (0: 64) */
    int32_t max_inflight;         /* batches on the GPU at once, 1..3 (0: 2) */
    int32_t max_batch_jobs;       /* jobs per batch (0: all pending) */
    int32_t serialized;           /* 1: sim and render on one stream, no overlap */
} vuda_serve_opts;
typedef struct {
    uint64_t req_id;
    int64_t job_id;
    int32_t status;               /* VUDA_OK, VUDA_ERR_BUSY (cancelled), or the admission error */
    int64_t step;                 /* the job's step index this request computed */
    double t_submit_ms, t_start_ms, t_done_ms;   /* host steady clock */
} vuda_result;
typedef struct {
    int32_t jobs, admitted, waiting, inflight;
    int64_t iterations, requests_done;
    double mean_batch;            /* jobs per launched batch */
    int32_t max_batch;
    int64_t used_bytes, peak_bytes;
} vuda_serve_stats;

vuda_status vuda_serve_create(const vuda_serve_opts* opts, vuda_server_t* out);
vuda_status vuda_serve_destroy(vuda_server_t server);
/* Queue a job for admission (the scene is copied).  VUDA_ERR_OOM if the job
 * alone exceeds the budget. */
vuda_status vuda_serve_add_job(vuda_server_t server, const vuda_scene* scene, const vuda_sim_params* params,
                               int64_t* job_id);
/* Request one step + render of the job; requests of a job run in order. */
vuda_status vuda_serve_submit(vuda_server_t server, int64_t job_id, uint64_t* req_id);
/* Completed requests (up to max), waiting up to wait_ms for the first.
 * With wait_ms > 0, VUDA_ERR_TIMEOUT (and *n = 0) when none completed in
 * that time; with wait_ms <= 0 it returns at once, VUDA_OK even if *n = 0. */
vuda_status vuda_serve_poll(vuda_server_t server, vuda_result* out, int32_t max, int32_t* n, int32_t wait_ms);
/* Cancel the job's queued requests and free it once its running ones finish. */
vuda_status vuda_serve_remove_job(vuda_server_t server, int64_t job_id);
/* The job's environment handle and frame (for reading results; call while
 * the job has no request queued or running).  VUDA_ERR_BUSY if not admitted. */
vuda_status vuda_serve_job_env(vuda_server_t server, int64_t job_id, vuda_env_t* env, vuda_frame* frame);
vuda_status vuda_serve_stats_get(vuda_server_t server, vuda_serve_stats* out);
/* Copy the job's last frame to host memory (rgb[P][3], depth[P], triid[P];
 * any may be NULL).  The job must be idle (VUDA_ERR_BUSY otherwise). */
vuda_status vuda_serve_read_frame(vuda_server_t server, int64_t job_id, uint8_t* rgb, float* depth, uint32_t* triid);

/* Physics step that allocates no device memory, for callers that cannot
 * allocate: code running inside a graph or stream region it does not own,
 * plug-ins handed a fixed device arena by their host application, processes
 * whose allocator belongs to another runtime.  The paper has no counterpart;
 * the arithmetic is exactly vuda_sim_step's.
 *   All arrays are caller-owned device memory with the layouts of vuda_scene
 *   (body_off[E+1], SoA planes of length num_bodies); pos/quat/vel/angvel are
 *   updated in place; pose[7][B] receives the final pose (xyz, wxyz);
 *   flags[E] receives VUDA_FLAG_CONTACT_OVERFLOW bits by OR (clear it first);
 *   ncontacts[E] the contact count of the last substep; force may be NULL.
 *   max_bodies (> 0 when num_envs > 0, else VUDA_ERR_INVALID) bounds
 *   body_off[e+1] - body_off[e]; smem_per_env 0 = default.  The kernel checks
 *   every environment's range against 0 <= body_off[e] <= body_off[e+1] <=
 *   num_bodies and body_off[e+1] - body_off[e] <= max_bodies before touching
 *   shared memory or the scratch; an environment that fails is skipped and
 *   gets VUDA_FLAG_BAD_RANGE in flags[e].
 * Scratch (contact spill records and their per-environment offsets) lives in
 * one fixed 16 MiB device array inside the library, held by every device that
 * loads it until the process exits.  Batches needing more scratch
 * (4 bytes x (2 (E + 1) rounded up to 64 + 36 x max_contacts_per_body x B))
 * are rejected with VUDA_ERR_INVALID before anything is launched.  The first
 * call on a device resolves the array's device address; make that first call
 * before any stream capture.  The address is cached per device for the rest
 * of the process: call with the device's primary context current (the CUDA
 * runtime's default; not inside another context such as a green context),
 * and not after a cudaDeviceReset of that device.  Every call shares the array: calls whose work
 * overlaps on the GPU (different streams, or different host threads) race and
 * must be serialised by the caller.  Async on `stream`. */
vuda_status vuda_sim_step_noalloc(int32_t num_envs, int32_t num_bodies, int32_t max_bodies, const int32_t* body_off,
                                  float* pos, float* quat, float* vel, float* angvel, const uint8_t* shape_type,
                                  const float* shape_dims, const float* inv_mass, const float* inv_inertia,
                                  const float* force, const vuda_sim_params* params, int32_t nsteps, float* pose,
                                  uint32_t* flags, int32_t* ncontacts, int32_t smem_per_env, vuda_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* VUDA_H */
