// Tiled render path: the rasteriser of render.cu split so that no work is
// repeated across a camera's image (the band kernel transforms and sets up
// every triangle of the environment once per band of rows).
//
//   bin_kernel, one CTA per camera: for each chunk of the environment's
//   bodies (ground quad first), transform and project the chunk's vertices
//   into shared memory, then set up every triangle once -- signed area (back
//   faces and degenerate triangles culled), bounding box clipped to the
//   image, edge functions and top-left bits -- and write it as an 80-byte
//   record to the camera's scratch area in global memory (read back by the
//   raster kernel from L2).  A counting sort in shared memory lists each
//   record that overlaps at most `nlim` (the bin limit) T x T tiles under
//   every one of them; records over more tiles go to one wide list of the
//   camera.
//   tile_kernel, one warp per tile and no CTA barriers.  The warp covers its
//   tile in strips of at most 256 pixels (8 x 8 tiles: one strip, 2 pixels a
//   lane; 16 x 16: one strip, 8 a lane; 32 x 32: four 32 x 8 strips, 8 a
//   lane), each strip a pass over the tile's lists: records whose unclipped
//   bounding box has at most kLanePx pixel centres are rasterised row by row
//   with 32-bit edge functions (exact for boxes that small), the rows of a
//   batch of 32 records dealt to the lanes in turn, into the warp's strip
//   key buffer in shared memory (atomicMin); larger records and
//   the wide list go through the warp-wide pass, in which every lane keeps
//   the keys of its run of pixels in registers.  The strip is then resolved
//   from min(register key, shared key) to RGB8, FP32 depth and u32 triangle
//   id.
// The tile size T (8, 16, 32) and the bin limit are the raster parameters
// the autotuner chooses between; every choice gives the same frames.
// Coverage rule, depth and key are those of the band kernel (integer edge
// functions at pixel centres with the top-left rule, depth
// area2 / (E0/z0 + E1/z1 + E2/z2), minimum of depth_bits << 32 | id), and the
// minimum does not depend on the order of the fragments, so both paths give
// identical frames.
#include <cuda_runtime.h>

#include <cstddef>

#include "internal.cuh"
#include "raster.cuh"

namespace vuda {
namespace {

constexpr int kBT = 256;          // bin_kernel threads
constexpr int kSieveCap = 2048;   // triangles per window of the bin kernel's sieve
constexpr int kNarrowTiles = 9;   // default bin limit: records over more tiles go to the camera's wide list
constexpr int kMaxBinLimit = 64;  // largest bin limit accepted
constexpr int kMaxTiles = 2048;   // tiles per camera the counting sort holds in shared memory (640 x 480: 1200)
constexpr int kLanePx = 64;       // unclipped bounding-box pixels up to which a record takes the 32-bit row path

// Geometry of one warp's T x T tile: strips of SH rows, R pixels per lane
// (LPR lanes per strip row), TW tiles (warps) per tile_kernel CTA.  Two
// warps per CTA: the warps of a CTA finish their tiles at different times
// (tiles hold different numbers of triangles) and the CTA's slot is freed
// only with its last warp, so small CTAs keep more warps resident (16 CTAs
// of 64 registers per thread fill an SM's register file).
template <int T>
struct TileGeom {
    static constexpr int SH = T * T > 256 ? 256 / T : T;
    static constexpr int R = T * SH / 32;
    static constexpr int LPR = T / R;
    static constexpr int STRIPS = T / SH;
    static constexpr int TW = 2;
    static_assert(LPR * SH == 32 && STRIPS * SH == T, "tile geometry");
};
constexpr unsigned kFullMask = 0xffffffffu;
constexpr unsigned kSmallBit = 8u;  // TriRec::tl bit: the record takes the 32-bit row path

// A set-up triangle, vertices oriented to positive area (80 bytes, 16-byte
// aligned in the scratch array).
struct __align__(16) TriRec {
    // edge i: E_i = A_i x + B_i y + C_i in 1/256 px, |A|, |B| <= 2^23.  C
    // holds C_i - b_i with b_i = 1 where edge i does not own its pixels (top-
    // left rule), so that a pixel centre is inside iff every biased value
    // E_i - b_i is >= 0; E_i itself (for the depth) is the biased value + b_i.
    int A[3], B[3];
    long long C[3];
    float iz[3];           // 1 / view depth of the vertices
    float af;              // (float) doubled area
    short x0, x1, y0, y1;  // pixel bounding box, clipped to the image
    uint32_t id;           // env-local triangle id
    unsigned tl;           // bits 0..2: edge i owns its pixels (top-left rule); kSmallBit
};
static_assert(sizeof(TriRec) == 80, "TriRec layout");

__device__ __forceinline__ TriRec load_rec(const TriRec* __restrict__ p) {
    union {
        int4 v[5];
        TriRec t;
    } u;
    const int4* q = reinterpret_cast<const int4*>(p);
#pragma unroll
    for (int k = 0; k < 5; k++) u.v[k] = __ldg(q + k);
    return u.t;
}

__device__ __forceinline__ void store_rec(TriRec* p, const TriRec& t) {
    union {
        int4 v[5];
        TriRec t;
    } u;
    u.t = t;
    int4* q = reinterpret_cast<int4*>(p);
#pragma unroll
    for (int k = 0; k < 5; k++) q[k] = u.v[k];
}

__device__ __forceinline__ TileItem load_item(const TileItem* __restrict__ p) {
    union {
        int4 v[5];
        TileItem t;
    } u;
    const int4* q = reinterpret_cast<const int4*>(p);
#pragma unroll
    for (int k = 0; k < 5; k++) u.v[k] = __ldg(q + k);
    return u.t;
}
static_assert(sizeof(TileItem) == 80 && offsetof(TileItem, rec_base) == 32 && offsetof(TileItem, toff_base) == 48 &&
                  offsetof(TileItem, pix_off) == 64 && offsetof(TileItem, col_base) == 72,
              "TileItem layout");

// Exclusive prefix sum over the kBT threads of the CTA, in thread order.
__device__ __forceinline__ int cta_excl_scan(int v, int* wsum, int& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFullMask, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    int off = 0;
    total = 0;
#pragma unroll
    for (int k = 0; k < kBT / 32; k++) {
        int s = wsum[k];
        if (k < w) off += s;
        total += s;
    }
    __syncthreads();
    return off + x - v;
}

// Set-up, shading and binning of camera `ci` of batch b (pose: its pose
// slot), by the whole CTA.
template <int T, bool kSieve>
__device__ __forceinline__ void bin_camera(const DevBatch& b, const float* __restrict__ pose, const TileScratch& ts,
                                           const TileItem& ci, int nlim) {
    __shared__ int vX[kVertexCache], vY[kVertexCache], vflag[kVertexCache];
    __shared__ float viz[kVertexCache];
    __shared__ float vW[kVertexCache][3];   // world positions, for the flat colours
    __shared__ int s_cnt[kMaxTiles];
    __shared__ int s_wsum[kBT / 32];
    __shared__ int s_nrec, s_nwide;
    __shared__ unsigned s_flags;
    __shared__ unsigned short s_q[kSieve ? kSieveCap : 1];   // the sieve's kept triangles (window-relative)
    __shared__ int s_nq;

    const int cam = ci.cam, e = ci.env;
    const int W = ci.W, H = ci.H;
    const int tiles_x = ci.tiles_x, ntiles = ci.ntiles;
    TriRec* rec = reinterpret_cast<TriRec*>(ts.rec) + ci.rec_base;
    uint32_t* wide = ts.wide + ci.rec_base;
    uint32_t* ent = ts.ent + ci.ent_base;
    int32_t* toff = ts.toff + ci.toff_base;
    const CamView cv = load_cam(b, cam);
    const int b0 = b.body_off[e];
    uint32_t* colors = b.tri_color + ci.col_base;
    const int rec_cap = (int)ci.rec_cap;

    for (int i = threadIdx.x; i < ntiles; i += kBT) s_cnt[i] = 0;
    if (threadIdx.x == 0) {
        s_nrec = 0;
        s_nwide = 0;
        s_flags = 0u;
        s_nq = 0;
    }
    for (int ck = b.chunk_off[e]; ck < b.chunk_off[e + 1]; ck++) {
        const int cb0 = b.chunk_lo[ck];   // env-local first body, -1 = ground
        const int nv = b.chunk_nv[ck], nt = b.chunk_nt[ck];
        const int2* vt = b.vtab + b.chunk_vtab[ck];
        const uint2* tt = b.ttab + b.chunk_ttab[ck];
        const uint32_t tri0 = (uint32_t)b.chunk_tri0[ck];
        __syncthreads();  // counters set; the previous chunk is done with the vertex cache
        for (int v = threadIdx.x; v < nv; v += kBT) {
            int X = 0, Y = 0;
            float iz = 0.0f, wx, wy, wz;
            vflag[v] = project_vertex(b, pose, cv, b0, cb0, vt[v], X, Y, iz, wx, wy, wz);
            vX[v] = X;
            vY[v] = Y;
            viz[v] = iz;
            vW[v][0] = wx;
            vW[v][1] = wy;
            vW[v][2] = wz;
        }
        __syncthreads();
        // set-up, shading and binning of triangle t of the chunk
        auto triangle = [&](int t) {
            const uint2 tv = tt[t];
            const int i0 = tv.x & 0xffff, i1 = tv.x >> 16, i2 = tv.y;
            const uint32_t id = tri0 + (uint32_t)t;
            // set-up, record, flat colour and binning of one screen triangle
            // (snapped vertices in mesh order) with the triangle's id
            auto emit = [&](int X0, int X1, int X2, int Y0, int Y1, int Y2, float z0, float z1, float z2) {
                const int mnx = min(X0, min(X1, X2)), mxx = max(X0, max(X1, X2));
                const int mny = min(Y0, min(Y1, Y2)), mxy = max(Y0, max(Y1, Y2));
                // pixel centres 256 p + 128 inside [mn, mx], before and after clipping to the image
                const int ux0 = (mnx - 128 + 255) >> 8, ux1 = (mxx - 128) >> 8;
                const int uy0 = (mny - 128 + 255) >> 8, uy1 = (mxy - 128) >> 8;
                const int px0 = max(ux0, 0), px1 = min(ux1, W - 1);
                const int py0 = max(uy0, 0), py1 = min(uy1, H - 1);
                if (px0 > px1 || py0 > py1) return;
                const long long area2 =
                    ((long long)X1 - X0) * ((long long)Y2 - Y0) - ((long long)Y1 - Y0) * ((long long)X2 - X0);
                if (area2 >= 0) return;   // back-facing or degenerate
                // oriented to positive area: (v0, v2, v1)
                const int X[3] = {X0, X2, X1}, Y[3] = {Y0, Y2, Y1};
                TriRec g;
                unsigned tl = 0u;
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    const int j = i == 2 ? 0 : i + 1, k = i == 0 ? 2 : i - 1;
                    const long long A = (long long)Y[j] - Y[k];
                    const long long Bv = (long long)X[k] - X[j];
                    g.A[i] = (int)A;
                    g.B[i] = (int)Bv;
                    const bool owns = (A > 0) || (A == 0 && Bv > 0);
                    g.C[i] = -A * X[j] - Bv * Y[j] - (owns ? 0 : 1);
                    if (owns) tl |= 1u << i;
                }
                const long long pa = ((long long)X[1] - X[0]) * ((long long)Y[2] - Y[0]) -
                                     ((long long)Y[1] - Y[0]) * ((long long)X[2] - X[0]);
                g.af = i64_to_f32(pa);
                g.iz[0] = z0;
                g.iz[1] = z2;
                g.iz[2] = z1;
                g.id = id;
                g.x0 = (short)px0; g.x1 = (short)px1; g.y0 = (short)py0; g.y1 = (short)py1;
                if ((long long)(ux1 - ux0 + 1) * (uy1 - uy0 + 1) <= kLanePx) tl |= kSmallBit;
                g.tl = tl;
                const int r = atomicAdd(&s_nrec, 1);
                if (r >= rec_cap) {   // reachable only through the extra fan triangles of clipping
                    atomicOr(&s_flags, (unsigned)VUDA_FLAG_CLIP_CAPACITY);
                    return;
                }
                store_rec(rec + r, g);
                // flat colour of the recorded triangle (only recorded triangles
                // can be the nearest at a pixel); the cameras of one environment
                // write the same value
                {
                    const int bi = cb0 + vt[i0].y;
                    const uint32_t alb = bi < 0 ? b.ground_albedo : __ldg(b.albedo + b0 + bi);
                    colors[id] = flat_color(vW[i0], vW[i1], vW[i2], alb, b.light);
                }
                const int tx0 = px0 / T, tx1 = px1 / T, ty0 = py0 / T, ty1 = py1 / T;
                if ((tx1 - tx0 + 1) * (ty1 - ty0 + 1) <= nlim) {
                    for (int ty = ty0; ty <= ty1; ty++)
                        for (int tx = tx0; tx <= tx1; tx++) atomicAdd(&s_cnt[ty * tiles_x + tx], 1);
                } else {
                    wide[atomicAdd(&s_nwide, 1)] = (uint32_t)r;
                }
            };
            const int fl = vflag[i0] | vflag[i1] | vflag[i2];
            if (fl == 0) {
                emit(vX[i0], vX[i1], vX[i2], vY[i0], vY[i1], vY[i2], viz[i0], viz[i1], viz[i2]);
            } else {
                // before the near plane or beyond the guard band: cull, clip or flag
                ClipFan f;
                const int cf = clip_near_fan(b, pose, cv, b0, cb0, vt[i0], vt[i1], vt[i2], f);
                if (cf) atomicOr(&s_flags, (unsigned)cf);
                for (int k = 0; k < f.n; k++)
                    emit(f.X[k][0], f.X[k][1], f.X[k][2], f.Y[k][0], f.Y[k][1], f.Y[k][2], f.iz[k][0], f.iz[k][1],
                         f.iz[k][2]);
            }
        };
        if constexpr (kSieve) {
            // fine meshes: most triangles cover no pixel centre or face away.
            // A first pass keeps the triangles that can leave a record (the
            // tests that open the set-up, or a vertex to clip), a second pass
            // runs the set-up on them with full warps; windows of kSieveCap.
            const int lane = threadIdx.x & 31;
            for (int w0 = 0; w0 < nt; w0 += kSieveCap) {
                const int w1 = min(nt, w0 + kSieveCap);
                for (int r0 = w0; r0 < w1; r0 += kBT) {
                    const int t = r0 + threadIdx.x;
                    bool keep = false;
                    if (t < w1) {
                        const uint2 tv = tt[t];
                        const int i0 = tv.x & 0xffff, i1 = tv.x >> 16, i2 = tv.y;
                        if (vflag[i0] | vflag[i1] | vflag[i2]) {
                            keep = true;
                        } else {
                            const int X0 = vX[i0], X1 = vX[i1], X2 = vX[i2], Y0 = vY[i0], Y1 = vY[i1], Y2 = vY[i2];
                            const int mnx = min(X0, min(X1, X2)), mxx = max(X0, max(X1, X2));
                            const int mny = min(Y0, min(Y1, Y2)), mxy = max(Y0, max(Y1, Y2));
                            const int px0 = max((mnx - 128 + 255) >> 8, 0), px1 = min((mxx - 128) >> 8, W - 1);
                            const int py0 = max((mny - 128 + 255) >> 8, 0), py1 = min((mxy - 128) >> 8, H - 1);
                            const long long area2 = ((long long)X1 - X0) * ((long long)Y2 - Y0) -
                                                    ((long long)Y1 - Y0) * ((long long)X2 - X0);
                            keep = px0 <= px1 && py0 <= py1 && area2 < 0;
                        }
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, keep);
                    int base = 0;
                    if (lane == 0 && m) base = atomicAdd(&s_nq, __popc(m));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (keep) s_q[base + __popc(m & ((1u << lane) - 1u))] = (unsigned short)(t - w0);
                }
                __syncthreads();
                const int nq = s_nq;
                for (int q = threadIdx.x; q < nq; q += kBT) triangle(w0 + s_q[q]);
                __syncthreads();   // the queue is read
                if (threadIdx.x == 0) s_nq = 0;
                __syncthreads();
            }
        } else {
            for (int t = threadIdx.x; t < nt; t += kBT) triangle(t);
        }
    }
    __syncthreads();
    // list offsets: exclusive prefix sum of the tile counts (at most kMaxTiles / kBT tiles per thread)
    const int per = (ntiles + kBT - 1) / kBT;
    const int i0 = threadIdx.x * per;
    int loc[kMaxTiles / kBT];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kMaxTiles / kBT; k++) {
        loc[k] = sum;
        if (k < per && i0 + k < ntiles) sum += s_cnt[i0 + k];
    }
    int total;
    const int off = cta_excl_scan(sum, s_wsum, total);   // its barriers order the reads above
#pragma unroll
    for (int k = 0; k < kMaxTiles / kBT; k++)
        if (k < per && i0 + k < ntiles) {
            s_cnt[i0 + k] = off + loc[k];   // becomes the fill cursor of the tile
            toff[i0 + k] = off + loc[k];
        }
    if (threadIdx.x == 0) {
        toff[ntiles] = total;
        toff[ntiles + 1] = s_nwide;
    }
    __syncthreads();
    // fill the tile lists (the order inside a list is free: the key minimum does not depend on it)
    const int nrec = min(s_nrec, rec_cap);
    for (int r = threadIdx.x; r < nrec; r += kBT) {
        const int2 bb = *reinterpret_cast<const int2*>(reinterpret_cast<const char*>(rec + r) + 64);
        const int px0 = (short)(bb.x & 0xffff), px1 = bb.x >> 16;
        const int py0 = (short)(bb.y & 0xffff), py1 = bb.y >> 16;
        const int tx0 = px0 / T, tx1 = px1 / T, ty0 = py0 / T, ty1 = py1 / T;
        if ((tx1 - tx0 + 1) * (ty1 - ty0 + 1) <= nlim) {
            for (int ty = ty0; ty <= ty1; ty++)
                for (int tx = tx0; tx <= tx1; tx++) ent[atomicAdd(&s_cnt[ty * tiles_x + tx], 1)] = (uint32_t)r;
        }
    }
    if (threadIdx.x == 0 && s_flags) atomicOr(b.flags + e, s_flags);
}

template <int T, bool kSieve>
__global__ void __launch_bounds__(kBT, 4) bin_kernel(DevBatch b, const float* __restrict__ pose, TileScratch ts,
                                                  const TileItem* __restrict__ cams, int nlim) {
    bin_camera<T, kSieve>(b, pose, ts, load_item(cams + blockIdx.x), nlim);
}

// The job of work-list position k: the last job whose first position
// (cam0, or item0 when `items`) is <= k.  Uniform across the calling threads.
__device__ __forceinline__ int find_job(const TiledJob* __restrict__ jobs, int njobs, int k, bool items) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int first = items ? __ldg(&jobs[mid].item0) : __ldg(&jobs[mid].cam0);
        if (first <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Work-list form: CTA k sets up camera k of the list; its job's batch
// descriptor is copied to shared memory.
template <int T>
__global__ void __launch_bounds__(kBT, 4) bin_list_kernel(const DevBatch* __restrict__ descs,
                                                       const TiledJob* __restrict__ jobs, int njobs, int nlim) {
    __shared__ DevBatch sd;
    const int jb = find_job(jobs, njobs, blockIdx.x, false);
    const int tag = __ldg(&jobs[jb].tag);
    const TileItem ci = load_item(jobs[jb].cams + (blockIdx.x - __ldg(&jobs[jb].cam0)));
    const int* src = reinterpret_cast<const int*>(descs + (tag & kItemDescMask));
    int* dst = reinterpret_cast<int*>(&sd);
    for (int k = threadIdx.x; k < (int)(sizeof(DevBatch) / 4); k += kBT) dst[k] = src[k];
    __syncthreads();
    const TileScratch ts = jobs[jb].ts;
    bin_camera<T, false>(sd, sd.pose[(tag >> 24) & 1], ts, ci, nlim);
}

// Row set-up of a small record for the dealt raster below: the biased edge
// values at the first pixel centre (x0, y0) of the record's clipped box,
// their steps along x and y, and the record's depth constants, in the
// lane's slot of the warp (four 16-byte groups, one array per group).  A
// small record's unclipped bounding box has at most kLanePx pixel centres,
// so its vertex spans and |A|, |B| stay below 65 x 256 < 2^14.1 and every
// edge value at a pixel centre of the box (or one step past it) below 2^30:
// 32-bit integers hold them exactly, and their float conversions are the
// correctly rounded ones.
struct RowSlots {
    int4* e;     // [32] E0, E1, E2 at (x0, y0); triangle id
    int4* dx;    // [32] x steps; x0 - tx0 | (x1 - tx0) << 8
    int4* dy;    // [32] y steps; bias bits | (y0 - sy0) << 3
    float4* z;   // [32] 1 / z of the vertices; doubled area
    int* first;  // [32] the batch's unit index of the record's first row
};

__device__ __forceinline__ void put_row_slot(const RowSlots& rs, int lane, const TriRec& t, int x0, int x1, int y0,
                                             int tx0, int sy0) {
    const long long cx = 256LL * x0 + 128, cy = 256LL * y0 + 128;
    const int R0 = (int)((long long)t.A[0] * cx + (long long)t.B[0] * cy + t.C[0]);
    const int R1 = (int)((long long)t.A[1] * cx + (long long)t.B[1] * cy + t.C[1]);
    const int R2 = (int)((long long)t.A[2] * cx + (long long)t.B[2] * cy + t.C[2]);
    rs.e[lane] = make_int4(R0, R1, R2, (int)t.id);
    rs.dx[lane] = make_int4(t.A[0] * 256, t.A[1] * 256, t.A[2] * 256, (x0 - tx0) | ((x1 - tx0) << 8));
    rs.dy[lane] = make_int4(t.B[0] * 256, t.B[1] * 256, t.B[2] * 256,
                            (int)((~t.tl) & 7u) | ((y0 - sy0) << 3));
    rs.z[lane] = make_float4(t.iz[0], t.iz[1], t.iz[2], t.af);
}

// Rasterises row r of a small record's clipped box from its slot (owner
// lane o; u is the row's unit index in the batch) into the warp's shared
// key buffer (atomicMin): the coverage test, depth and key of the warp-wide
// pass in 32-bit arithmetic, so the keys do not depend on how the rows are
// dealt.
template <int T>
__device__ __forceinline__ void slot_row(const RowSlots& rs, int o, int u, int tx0, unsigned long long* sk) {
    const int4 e = rs.e[o], dx = rs.dx[o], dy = rs.dy[o];
    const float4 z = rs.z[o];
    const int r = u - rs.first[o];
    const int xa = dx.w & 255, xb = (dx.w >> 8) & 255;
    int E0 = e.x + r * dy.x, E1 = e.y + r * dy.y, E2 = e.z + r * dy.z;
    const int b0 = dy.w & 1, b1 = (dy.w >> 1) & 1, b2 = (dy.w >> 2) & 1;
    unsigned long long* row = sk + ((dy.w >> 3) + r) * T;
    for (int px = xa; px <= xb; px++) {
        if ((E0 | E1 | E2) >= 0) {
            const float den = (__int2float_rn(E0 + b0) * z.x + __int2float_rn(E1 + b1) * z.y) +
                              __int2float_rn(E2 + b2) * z.z;
            const float depth = z.w / den;
            atomicMin(row + px, ((unsigned long long)__float_as_uint(depth) << 32) | (uint32_t)e.w);
        }
        E0 += dx.x;
        E1 += dx.y;
        E2 += dx.z;
    }
}

// Warp-wide pass of one record over the strip: the lane tests its run of
// nx <= R pixels (row y, columns xs ..) with 64-bit edge functions and keeps
// the minimum keys in registers.  The record address is the same in all
// lanes.
template <int R>
__device__ __forceinline__ void warp_pass(const TriRec* __restrict__ p, int y, int xs, int nx,
                                          unsigned long long* key) {
    const TriRec t = load_rec(p);
    if (nx <= 0 || y < t.y0 || y > t.y1 || xs + nx - 1 < t.x0 || xs > t.x1) return;
    const long long cy = 256LL * y + 128;
    const long long cx = 256LL * xs + 128;
    long long E0 = (long long)t.A[0] * cx + (long long)t.B[0] * cy + t.C[0];
    long long E1 = (long long)t.A[1] * cx + (long long)t.B[1] * cy + t.C[1];
    long long E2 = (long long)t.A[2] * cx + (long long)t.B[2] * cy + t.C[2];
    const long long d0 = 256LL * t.A[0], d1 = 256LL * t.A[1], d2 = 256LL * t.A[2];
    // the (biased) edge functions are affine along the run: negative at both
    // of its ends for one edge means no pixel of the run is covered
    const long long m = nx - 1;
    if ((E0 < 0 && E0 + m * d0 < 0) || (E1 < 0 && E1 + m * d1 < 0) || (E2 < 0 && E2 + m * d2 < 0)) return;
#pragma unroll
    for (int k = 0; k < R; k++) {
        // inside iff every biased edge value is >= 0: the sign of the OR of their high words
        const int hi = (int)(((unsigned long long)E0 | (unsigned long long)E1 | (unsigned long long)E2) >> 32);
        if (k < nx && hi >= 0) {
            const unsigned nb = ~t.tl;   // bias bits b_i
            const float den = (i64_to_f32(E0 + (long long)(nb & 1u)) * t.iz[0] +
                               i64_to_f32(E1 + (long long)((nb >> 1) & 1u)) * t.iz[1]) +
                              i64_to_f32(E2 + (long long)((nb >> 2) & 1u)) * t.iz[2];
            const float depth = t.af / den;
            const unsigned long long kk = ((unsigned long long)__float_as_uint(depth) << 32) | t.id;
            key[k] = kk < key[k] ? kk : key[k];
        }
        E0 += d0;
        E1 += d1;
        E2 += d2;
    }
}

// Resolve a lane's run of nx <= R pixels starting at frame pixel p0 from
// its keys to depth, triangle id and RGB8.  Full runs go out as streaming
// vector stores (the frame is not read again on the device, and evict-first
// stores keep the L2 for the triangle records still to be read).
template <int R>
__device__ __forceinline__ void resolve_run(const unsigned long long* key, int nx, int64_t p0,
                                            const uint32_t* __restrict__ colors, const vuda_frame& fr) {
    float d[R];
    uint32_t tid[R], col[R];
#pragma unroll
    for (int k = 0; k < R; k++) {
        const unsigned long long kk = key[k];
        if (kk == ~0ULL) {
            d[k] = 0.0f;
            tid[k] = 0xFFFFFFFFu;
            col[k] = 0u;
        } else {
            tid[k] = (uint32_t)(kk & 0xFFFFFFFFull);
            d[k] = __uint_as_float((uint32_t)(kk >> 32));
            col[k] = k < nx ? __ldg(colors + tid[k]) : 0u;
        }
    }
    if (R == 8) {
        const bool vec = nx == 8 && ((reinterpret_cast<uintptr_t>(fr.depth + p0) & 15) == 0) &&
                         ((reinterpret_cast<uintptr_t>(fr.rgb + 3 * p0) & 7) == 0) &&
                         (!fr.triid || (reinterpret_cast<uintptr_t>(fr.triid + p0) & 15) == 0);
        if (vec) {
            float4* dp = reinterpret_cast<float4*>(fr.depth + p0);
            __stcs(dp, make_float4(d[0], d[1], d[2], d[3]));
            __stcs(dp + 1, make_float4(d[4], d[5], d[6], d[7]));
            if (fr.triid) {
                uint4* tp = reinterpret_cast<uint4*>(fr.triid + p0);
                __stcs(tp, make_uint4(tid[0], tid[1], tid[2], tid[3]));
                __stcs(tp + 1, make_uint4(tid[4], tid[5], tid[6], tid[7]));
            }
            // 8 pixels = 24 bytes = 6 words, little endian r g b r | g b r g | b r g b | ...,
            // written as three 8-byte stores (the run starts 8-byte aligned)
            uint32_t wd[6];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint32_t c0 = col[4 * h], c1 = col[4 * h + 1], c2 = col[4 * h + 2], c3 = col[4 * h + 3];
                wd[3 * h] = (c0 & 0xFFFFFFu) | ((c1 & 0xFFu) << 24);
                wd[3 * h + 1] = ((c1 >> 8) & 0xFFFFu) | ((c2 & 0xFFFFu) << 16);
                wd[3 * h + 2] = ((c2 >> 16) & 0xFFu) | ((c3 & 0xFFFFFFu) << 8);
            }
            uint2* r64 = reinterpret_cast<uint2*>(fr.rgb + 3 * p0);
#pragma unroll
            for (int q = 0; q < 3; q++) __stcs(r64 + q, make_uint2(wd[2 * q], wd[2 * q + 1]));
            return;
        }
    } else if (R == 2) {
        const bool vec = nx == 2 && ((reinterpret_cast<uintptr_t>(fr.depth + p0) & 7) == 0) &&
                         ((reinterpret_cast<uintptr_t>(fr.rgb + 3 * p0) & 1) == 0) &&
                         (!fr.triid || (reinterpret_cast<uintptr_t>(fr.triid + p0) & 7) == 0);
        if (vec) {
            __stcs(reinterpret_cast<float2*>(fr.depth + p0), make_float2(d[0], d[1]));
            if (fr.triid) __stcs(reinterpret_cast<uint2*>(fr.triid + p0), make_uint2(tid[0], tid[1]));
            // 2 pixels = 6 bytes r g | b r | g b, three 2-byte stores
            unsigned short* r16 = reinterpret_cast<unsigned short*>(fr.rgb + 3 * p0);
            __stcs(r16, (unsigned short)(col[0] & 0xFFFFu));
            __stcs(r16 + 1, (unsigned short)(((col[0] >> 16) & 0xFFu) | ((col[1] & 0xFFu) << 8)));
            __stcs(r16 + 2, (unsigned short)((col[1] >> 8) & 0xFFFFu));
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < R; k++)
        if (k < nx) {
            fr.depth[p0 + k] = d[k];
            if (fr.triid) fr.triid[p0 + k] = tid[k];
            fr.rgb[3 * (p0 + k)] = col[k] & 255u;
            fr.rgb[3 * (p0 + k) + 1] = (col[k] >> 8) & 255u;
            fr.rgb[3 * (p0 + k) + 2] = (col[k] >> 16) & 255u;
        }
}

// Work item (camera, first tile): warp w rasterises and resolves tile
// first + w of the camera, one strip at a time.
template <int T>
__device__ __forceinline__ void tile_work(const uint32_t* __restrict__ tri_color, const TileScratch& ts,
                                          const vuda_frame& fr, const TileItem* __restrict__ itp) {
    using G = TileGeom<T>;
    constexpr int R = G::R;
    __shared__ unsigned long long s_key[G::TW][T * G::SH];
    __shared__ int s_big[G::TW][32];
    __shared__ int4 s_rs[G::TW][3][32];
    __shared__ float4 s_rz[G::TW][32];
    __shared__ int s_first[G::TW][32];
    __shared__ unsigned char s_own[G::TW][32 * G::SH];   // owner lane of each dealt row
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const RowSlots rs{s_rs[threadIdx.x >> 5][0], s_rs[threadIdx.x >> 5][1], s_rs[threadIdx.x >> 5][2],
                      s_rz[threadIdx.x >> 5], s_first[threadIdx.x >> 5]};
    const int4 geo = __ldg(reinterpret_cast<const int4*>(itp));        // cam, tile0, W, H
    const int2 tl2 = __ldg(reinterpret_cast<const int2*>(itp) + 2);    // tiles_x, ntiles
    const longlong2 rb = __ldg(reinterpret_cast<const longlong2*>(itp) + 2);   // rec_base, ent_base
    const long long toff_base = __ldg(reinterpret_cast<const long long*>(itp) + 6);
    const int tile = geo.y + w;
    const int W = geo.z, H = geo.w;
    const int tiles_x = tl2.x, ntiles = tl2.y;
    if (tile >= ntiles) return;   // whole warp; no CTA barrier follows
    const TriRec* __restrict__ rec = reinterpret_cast<const TriRec*>(ts.rec) + rb.x;
    const uint32_t* __restrict__ wide = ts.wide + rb.x;
    const uint32_t* __restrict__ ent = ts.ent + rb.y;
    const int32_t* __restrict__ toff = ts.toff + toff_base;
    const int tx0 = (tile % tiles_x) * T, ty0 = (tile / tiles_x) * T;
    const int tx1 = min(tx0 + T, W) - 1, ty1 = min(ty0 + T, H) - 1;
    unsigned long long* sk = s_key[w];
    const int beg = __ldg(toff + tile), end = __ldg(toff + tile + 1), nw = __ldg(toff + ntiles + 1);
#pragma unroll 1
    for (int st = 0; st < G::STRIPS; st++) {
        const int sy0 = ty0 + st * G::SH;
        if (sy0 > ty1) break;   // warp-uniform
        const int sy1 = min(sy0 + G::SH - 1, ty1);
        // lane: row lane / LPR of the strip, columns R (lane % LPR) .. + R - 1
        const int y = sy0 + lane / G::LPR, xs = tx0 + R * (lane % G::LPR);
        const int nx = y <= sy1 ? max(0, min(R, tx1 - xs + 1)) : 0;
        __syncwarp();   // the previous strip's resolve is done with the shared keys
#pragma unroll
        for (int k = 0; k < R; k++) sk[lane + 32 * k] = ~0ULL;
        __syncwarp();
        unsigned long long key[R];
#pragma unroll
        for (int k = 0; k < R; k++) key[k] = ~0ULL;

        for (int base = beg; base < end; base += 32) {
            const int i = base + lane;
            bool big = false;
            uint32_t r = 0;
            int nrow = 0;
            if (i < end) {
                r = __ldg(ent + i);
                const TriRec t = load_rec(rec + r);
                const int x0 = max((int)t.x0, tx0), x1 = min((int)t.x1, tx1);
                const int y0 = max((int)t.y0, sy0), y1 = min((int)t.y1, sy1);
                if (x0 <= x1 && y0 <= y1) {
                    if (t.tl & kSmallBit) {
                        nrow = y1 - y0 + 1;
                        put_row_slot(rs, lane, t, x0, x1, y0, tx0, sy0);
                    } else {
                        big = true;
                    }
                }
            }
            // the rows of the batch's small records are dealt to the lanes in
            // turn (row u of the batch to lane u % 32), so that the warp's
            // time is the batch's rows / 32 rather than its largest record
            int incl = nrow;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(kFullMask, incl, o);
                if (lane >= o) incl += v;
            }
            const int nunits = __shfl_sync(kFullMask, incl, 31);
            if (nunits > 0) {
                if (nrow > 0) {
                    rs.first[lane] = incl - nrow;
                    for (int k = incl - nrow; k < incl; k++) s_own[w][k] = (unsigned char)lane;
                }
                __syncwarp();
                for (int u = lane; u < nunits; u += 32) slot_row<T>(rs, s_own[w][u], u, tx0, sk);
                __syncwarp();   // the slots and owners are reused by the next batch
            }
            const unsigned m = __ballot_sync(kFullMask, big);
            if (big) s_big[w][__popc(m & ((1u << lane) - 1u))] = (int)r;
            __syncwarp();
            const int nb = __popc(m);
            for (int q = 0; q < nb; q++) warp_pass<R>(rec + s_big[w][q], y, xs, nx, key);
            __syncwarp();   // s_big is reused by the next batch
        }
        for (int q = 0; q < nw; q++) warp_pass<R>(rec + __ldg(wide + q), y, xs, nx, key);
        __syncwarp();       // the lanes' shared-memory keys are complete

        if (nx > 0) {
            const longlong2 pc = __ldg(reinterpret_cast<const longlong2*>(itp) + 4);   // pix_off, col_base
            const unsigned long long* sl = sk + (lane / G::LPR) * T + R * (lane % G::LPR);
#pragma unroll
            for (int k = 0; k < R; k++) {
                const unsigned long long kk = sl[k];
                key[k] = key[k] < kk ? key[k] : kk;
            }
            resolve_run<R>(key, nx, pc.x + (int64_t)y * W + xs, tri_color + pc.y, fr);
        }
    }
}

template <int T>
__global__ void __launch_bounds__(TileGeom<T>::TW * 32, 32 / TileGeom<T>::TW)
    tile_kernel(DevBatch b, TileScratch ts, vuda_frame fr, const TileItem* __restrict__ items) {
    tile_work<T>(b.tri_color, ts, fr, items + blockIdx.x);
}

// Work-list form: CTA k rasterises raster item k of the list; the frame,
// colour table and scratch are its job's batch's.
template <int T>
__global__ void __launch_bounds__(TileGeom<T>::TW * 32, 32 / TileGeom<T>::TW)
    tile_list_kernel(const DevBatch* __restrict__ descs, const TiledJob* __restrict__ jobs, int njobs) {
    const int jb = find_job(jobs, njobs, blockIdx.x, true);
    const TileItem* itp = jobs[jb].items + (blockIdx.x - __ldg(&jobs[jb].item0));
    const DevBatch* d = descs + (__ldg(&jobs[jb].tag) & kItemDescMask);
    const TileScratch ts = jobs[jb].ts;
    const vuda_frame fr = d->frame;
    tile_work<T>(d->tri_color, ts, fr, itp);
}

}  // namespace

int tiled_max_tiles() { return kMaxTiles; }
int tiled_default_tile() { return 16; }
int tiled_default_bin_limit() { return kNarrowTiles; }
int tiled_max_bin_limit() { return kMaxBinLimit; }
int tiled_tiles_per_item(int tile) {
    return tile == 8 ? TileGeom<8>::TW : tile == 32 ? TileGeom<32>::TW : TileGeom<16>::TW;
}
size_t tiled_record_bytes() { return sizeof(TriRec); }

template <int T>
static cudaError_t launch_tiled_t(const DevBatch& b, const float* pose, const vuda_frame& fr, const TileScratch& ts,
                                  const TileItem* cams, const TileItem* items, int nitems, int nlim, bool sieve,
                                  cudaStream_t stream) {
    if (sieve) bin_kernel<T, true><<<b.C, kBT, 0, stream>>>(b, pose, ts, cams, nlim);
    else bin_kernel<T, false><<<b.C, kBT, 0, stream>>>(b, pose, ts, cams, nlim);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || nitems == 0) return err;
    tile_kernel<T><<<nitems, TileGeom<T>::TW * 32, 0, stream>>>(b, ts, fr, items);
    return cudaGetLastError();
}

cudaError_t launch_render_tiled_list(const DevBatch* descs, const TiledJob* jobs, int njobs, int ncams, int nitems,
                                     cudaStream_t stream) {
    if (njobs == 0 || ncams == 0) return cudaSuccess;
    bin_list_kernel<16><<<ncams, kBT, 0, stream>>>(descs, jobs, njobs, kNarrowTiles);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || nitems == 0) return err;
    tile_list_kernel<16><<<nitems, TileGeom<16>::TW * 32, 0, stream>>>(descs, jobs, njobs);
    return cudaGetLastError();
}

cudaError_t launch_render_tiled(const DevBatch& b, const float* pose, const vuda_frame& fr, const TileScratch& ts,
                                const TileItem* cams, const TileItem* items, int nitems, int tile, int nlim, bool sieve,
                                cudaStream_t stream) {
    if (b.C == 0) return cudaSuccess;
    if (nlim < 1 || nlim > kMaxBinLimit) return cudaErrorInvalidValue;
    switch (tile) {
        case 8: return launch_tiled_t<8>(b, pose, fr, ts, cams, items, nitems, nlim, sieve, stream);
        case 16: return launch_tiled_t<16>(b, pose, fr, ts, cams, items, nitems, nlim, sieve, stream);
        case 32: return launch_tiled_t<32>(b, pose, fr, ts, cams, items, nitems, nlim, sieve, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace vuda
