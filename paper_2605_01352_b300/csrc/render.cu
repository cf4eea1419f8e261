// Batched per-environment camera render: a tile-binned fixed-point compute
// rasteriser (the rendering phase the paper runs through Vulkan's vertex ->
// rasterisation -> fragment pipeline, Sec. 2.1).
//
// Work item = (camera, band of rows).  One CTA of 256 threads per work item:
//   1. for each chunk of the env's bodies (ground quad first) whose vertices
//      fit the shared-memory vertex cache: transform every vertex
//      world = R(q) (s * v) + p, view = basis . (world - eye), project
//      sx = W/2 + fpy xc / zc, sy = H/2 - fpy yc / zc, snap to 24.8 fixed
//      point (round to nearest even).  Triangles crossing the near plane
//      (zc = 0.01) are clipped there (Sutherland-Hodgman, a fan of one or
//      two triangles with the original id); vertices beyond the 2^14 px
//      guard band invalidate their triangles (flagged).
//   2. one thread per triangle: integer signed area (back faces and
//      degenerate triangles culled), bounding box clipped to the band, flat
//      colour from the world face normal.  Triangles covering at most 16
//      bounding-box pixels are rasterised by their thread straight into the
//      shared-memory z-buffer (atomicMin); larger ones are recorded and
//      binned into 16 x 16 pixel tiles in shared memory.
//   3. tile pass: one warp per tile, each lane owns a run of 8 pixels and
//      keeps their keys in registers while it walks the tile's bin.
//   Coverage: 64-bit integer edge functions at pixel centres with the
//   top-left tie rule.  Depth: perspective-correct area2 / (E0/z0 + E1/z1 +
//   E2/z2).  Visibility: minimum of the 64-bit key depth_bits << 32 | id
//   (ties go to the lower triangle id).
//   4. resolve the band: RGB8 from the per-triangle colour table, FP32 depth,
//      u32 triangle id, written with 16-byte stores.
#include <cuda_runtime.h>

#include "internal.cuh"
#include "raster.cuh"

namespace vuda {
namespace {

constexpr int kRT = 256;           // threads per CTA
constexpr int kWarps = kRT / 32;
constexpr int kVcap = kVertexCache; // vertices per chunk
constexpr int kChunkBodies = 128;  // bodies per chunk
constexpr int kSmallPx = 16;       // triangles with at most this many bbox pixels stay thread-local
constexpr int kBigCap = 256;       // binned triangles per chunk pass
constexpr int kMaskWords = kBigCap / 32;

struct Tri {              // a visible, front-facing triangle, vertices oriented to positive area
    int X[3], Y[3];       // 24.8 fixed point
    float iz[3];
    uint32_t id;
    short x0, x1, y0, y1; // pixel bbox (inclusive), clipped to the band
};

struct Band {
    int W, y0, y1;          // rows [y0, y1)
    unsigned long long* z;  // keys of rows [y0, y1), row stride W
    unsigned* count;        // optional coverage counts
};

// Orients and bounds a snapped triangle.  Returns false if it is culled
// (back-facing / degenerate) or misses the band.
__device__ __forceinline__ bool setup_tri(const int* X, const int* Y, const float* iz, uint32_t id, const Band& bd,
                                          Tri& t) {
    int mnx = min(X[0], min(X[1], X[2])), mxx = max(X[0], max(X[1], X[2]));
    int mny = min(Y[0], min(Y[1], Y[2])), mxy = max(Y[0], max(Y[1], Y[2]));
    int px0 = (mnx - 128 + 255) >> 8, px1 = (mxx - 128) >> 8;
    int py0 = (mny - 128 + 255) >> 8, py1 = (mxy - 128) >> 8;
    px0 = max(px0, 0);
    px1 = min(px1, bd.W - 1);
    py0 = max(py0, bd.y0);
    py1 = min(py1, bd.y1 - 1);
    if (px0 > px1 || py0 > py1) return false;   // misses the band (cheap test first)
    long long x0 = X[0], y0 = Y[0], x1 = X[1], y1 = Y[1], x2 = X[2], y2 = Y[2];
    long long area2 = (x1 - x0) * (y2 - y0) - (y1 - y0) * (x2 - x0);
    if (area2 >= 0) return false;               // back-facing or degenerate
    t.X[0] = X[0]; t.Y[0] = Y[0]; t.iz[0] = iz[0];
    t.X[1] = X[2]; t.Y[1] = Y[2]; t.iz[1] = iz[2];
    t.X[2] = X[1]; t.Y[2] = Y[1]; t.iz[2] = iz[1];
    t.id = id;
    t.x0 = (short)px0; t.x1 = (short)px1; t.y0 = (short)py0; t.y1 = (short)py1;
    return true;
}

// Edge functions E_i = A_i x + B_i y + C_i (1/256 px) of a triangle.  C
// holds C_i - b_i with b_i = 1 where edge i does not own its pixels (top-left
// rule): a pixel centre is inside iff every biased value is >= 0, and E_i
// (for the depth) is the biased value + b_i.
struct Edges {
    long long A[3], B[3], C[3];
    bool tl[3];
    float af;
};

__device__ __forceinline__ void edges(const Tri& t, Edges& e) {
#pragma unroll
    for (int i = 0; i < 3; i++) {
        int j = i == 2 ? 0 : i + 1, k = i == 0 ? 2 : i - 1;
        long long A = (long long)t.Y[j] - t.Y[k];
        long long B = (long long)t.X[k] - t.X[j];
        e.A[i] = A;
        e.B[i] = B;
        e.tl[i] = (A > 0) || (A == 0 && B > 0);
        e.C[i] = -A * t.X[j] - B * t.Y[j] - (e.tl[i] ? 0 : 1);
    }
    long long area2 = ((long long)t.X[1] - t.X[0]) * ((long long)t.Y[2] - t.Y[0]) -
                      ((long long)t.Y[1] - t.Y[0]) * ((long long)t.X[2] - t.X[0]);
    e.af = i64_to_f32(area2);
}

// Biased edge values: inside iff all three are >= 0.
__device__ __forceinline__ bool inside(long long E0, long long E1, long long E2) { return (E0 | E1 | E2) >= 0; }

__device__ __forceinline__ unsigned long long frag_key(long long E0, long long E1, long long E2, const Tri& t,
                                                       const Edges& e) {
    float den = (i64_to_f32(E0 + (e.tl[0] ? 0 : 1)) * t.iz[0] + i64_to_f32(E1 + (e.tl[1] ? 0 : 1)) * t.iz[1]) +
                i64_to_f32(E2 + (e.tl[2] ? 0 : 1)) * t.iz[2];
    float depth = e.af / den;
    return ((unsigned long long)__float_as_uint(depth) << 32) | t.id;
}

// A binned triangle with its edge functions set up once, by the thread that
// submitted it, for all the lanes of the tile pass.
struct BigRec {
    int A[3], B[3];       // |A|, |B| < 2^23 inside the guard band
    long long C[3];       // biased as in Edges
    float iz[3];
    float af;             // (float) area2
    uint32_t id;
    short x0, x1, y0, y1;
    unsigned tl;          // bit i: edge i owns its pixels (b_i = 1 - bit i)
};

// One thread rasterises a small triangle into the shared-memory z-buffer.
__device__ __forceinline__ void raster_thread(const Tri& t, const Band& bd) {
    Edges e;
    edges(t, e);
    for (int py = t.y0; py <= t.y1; py++) {
        long long cy = 256LL * py + 128;
        long long cx = 256LL * t.x0 + 128;
        long long E0 = e.A[0] * cx + e.B[0] * cy + e.C[0];
        long long E1 = e.A[1] * cx + e.B[1] * cy + e.C[1];
        long long E2 = e.A[2] * cx + e.B[2] * cy + e.C[2];
        for (int px = t.x0; px <= t.x1; px++) {
            if (inside(E0, E1, E2)) {
                int o = (py - bd.y0) * bd.W + px;
                atomicMin(bd.z + o, frag_key(E0, E1, E2, t, e));
                if (bd.count) atomicAdd(bd.count + o, 1u);
            }
            E0 += e.A[0] * 256;
            E1 += e.A[1] * 256;
            E2 += e.A[2] * 256;
        }
    }
}

struct Bins {
    BigRec* rec;         // [kBigCap]
    int* nrec;
    unsigned* mask;      // [ntiles][kMaskWords]: bit r set if record r overlaps the tile
    int tiles_x, ntiles;
};

// Bin a recorded triangle into the tiles its bbox overlaps.
__device__ __forceinline__ void bin_tri(const Tri& t, int r, const Band& bd, Bins& bn) {
    int tx0 = t.x0 / kTile, tx1 = t.x1 / kTile;
    int ty0 = (t.y0 - bd.y0) / kTile, ty1 = (t.y1 - bd.y0) / kTile;
    for (int ty = ty0; ty <= ty1; ty++)
        for (int tx = tx0; tx <= tx1; tx++)
            atomicOr(bn.mask + (ty * bn.tiles_x + tx) * kMaskWords + (r >> 5), 1u << (r & 31));
}

// Tile pass: warp w walks tiles w, w + kWarps, ...; lane l owns pixels
// (row l / 2, columns 8 (l % 2) .. +7) of the tile and keeps their keys in
// registers while it walks the tile's records (any order: the key minimum
// does not depend on it).
__device__ void tile_pass(const Band& bd, const Bins& bn) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int tile = warp; tile < bn.ntiles; tile += kWarps) {
        const unsigned* m = bn.mask + tile * kMaskWords;
        unsigned any = 0;
#pragma unroll
        for (int w = 0; w < kMaskWords; w++) any |= m[w];
        if (!any) continue;
        int tx = tile % bn.tiles_x, ty = tile / bn.tiles_x;
        int y = bd.y0 + ty * kTile + (lane >> 1);
        int xs = tx * kTile + (lane & 1) * 8;
        bool rowok = y < bd.y1;
        int nx = rowok ? min(8, bd.W - xs) : 0;
        unsigned long long key[8];
        unsigned long long* zrow = bd.z + (size_t)(y - bd.y0) * bd.W + xs;
#pragma unroll
        for (int k = 0; k < 8; k++) key[k] = k < nx ? zrow[k] : ~0ULL;
        unsigned cnt8[8];
#pragma unroll
        for (int k = 0; k < 8; k++) cnt8[k] = 0;
        for (int w = 0; w < kMaskWords; w++) {
            unsigned bits = m[w];
            while (bits) {
                int r = (w << 5) + __ffs(bits) - 1;
                bits &= bits - 1;
                const BigRec& t = bn.rec[r];
                if (nx <= 0 || y < t.y0 || y > t.y1 || xs + nx - 1 < t.x0 || xs > t.x1) continue;
                const long long cy = 256LL * y + 128;
                const long long cx = 256LL * xs + 128;
                long long E0 = (long long)t.A[0] * cx + (long long)t.B[0] * cy + t.C[0];
                long long E1 = (long long)t.A[1] * cx + (long long)t.B[1] * cy + t.C[1];
                long long E2 = (long long)t.A[2] * cx + (long long)t.B[2] * cy + t.C[2];
                const long long d0 = 256LL * t.A[0], d1 = 256LL * t.A[1], d2 = 256LL * t.A[2];
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    // inside iff every biased edge value is >= 0: the sign of the OR of their high words
                    const int hi = (int)(((unsigned long long)E0 | (unsigned long long)E1 | (unsigned long long)E2) >> 32);
                    if (k < nx && hi >= 0) {
                        const unsigned nb = ~t.tl;   // bias bits b_i
                        float den = (i64_to_f32(E0 + (long long)(nb & 1u)) * t.iz[0] +
                                     i64_to_f32(E1 + (long long)((nb >> 1) & 1u)) * t.iz[1]) +
                                    i64_to_f32(E2 + (long long)((nb >> 2) & 1u)) * t.iz[2];
                        float depth = t.af / den;
                        unsigned long long kk = ((unsigned long long)__float_as_uint(depth) << 32) | t.id;
                        key[k] = kk < key[k] ? kk : key[k];
                        cnt8[k]++;
                    }
                    E0 += d0;
                    E1 += d1;
                    E2 += d2;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 8; k++)
            if (k < nx) {
                zrow[k] = key[k];
                if (bd.count) bd.count[(size_t)(y - bd.y0) * bd.W + xs + k] += cnt8[k];
            }
    }
}

__device__ __forceinline__ void init_band(const Band& bd) {
    int n = (bd.y1 - bd.y0) * bd.W;
    for (int i = threadIdx.x; i < n; i += kRT) {
        bd.z[i] = ~0ULL;
        if (bd.count) bd.count[i] = 0u;
    }
}

// A visible triangle goes to the small (thread-local) path or is recorded
// and binned; when the records are full it is rasterised by its thread
// (exact either way, only slower).
__device__ __forceinline__ void submit_tri(const Tri& t, const Band& bd, Bins& bn) {
    int npx = (t.x1 - t.x0 + 1) * (t.y1 - t.y0 + 1);
    if (npx > kSmallPx) {
        int r = atomicAdd(bn.nrec, 1);
        if (r < kBigCap) {
            Edges e;
            edges(t, e);
            BigRec& g = bn.rec[r];
#pragma unroll
            for (int i = 0; i < 3; i++) {
                g.A[i] = (int)e.A[i];
                g.B[i] = (int)e.B[i];
                g.C[i] = e.C[i];
                g.iz[i] = t.iz[i];
            }
            g.af = e.af;
            g.id = t.id;
            g.x0 = t.x0; g.x1 = t.x1; g.y0 = t.y0; g.y1 = t.y1;
            g.tl = (e.tl[0] ? 1u : 0u) | (e.tl[1] ? 2u : 0u) | (e.tl[2] ? 4u : 0u);
            bin_tri(t, r, bd, bn);
            return;
        }
    }
    raster_thread(t, bd);
}

// Rasterise the recorded triangles and clear the records.  Must be called by
// all threads of the CTA, after a barrier that follows the last submit_tri.
__device__ __forceinline__ void drain(const Band& bd, Bins& bn) {
    if (*bn.nrec > 0) {  // uniform after the barrier
        tile_pass(bd, bn);
        __syncthreads();
        for (int i = threadIdx.x; i < bn.ntiles * kMaskWords; i += kRT) bn.mask[i] = 0u;
        if (threadIdx.x == 0) *bn.nrec = 0;
        __syncthreads();
    }
}

struct RenderArgs {
    DevBatch b;
    const float* pose;       // [7][B]
    vuda_frame fr;
    const int32_t* item_cam; // [items]
    const int32_t* item_y0;  // [items]
    int band_rows, max_w;
};

__host__ __device__ inline int tiles_for(int rows, int W) {
    return ((rows + kTile - 1) / kTile) * ((W + kTile - 1) / kTile);
}

__host__ __device__ inline size_t render_smem_bytes(int band_rows, int W) {
    size_t s = (size_t)band_rows * W * 8;                        // z keys
    s += sizeof(BigRec) * kBigCap;                               // binned triangles
    s += (size_t)kVcap * (4 + 4 + 4 + 4);                        // vertex cache
    int nt = tiles_for(band_rows, W);
    s += (size_t)nt * kMaskWords * 4 + 16;                       // tile masks, counters
    return (s + 15) & ~(size_t)15;
}

// One (camera, band) work item by the whole CTA.  b lives in shared memory.
__device__ __forceinline__ void render_band(const DevBatch& b, int cam, int y0, const float* __restrict__ pose,
                                            const vuda_frame& fr, int band_rows, int max_w) {
    extern __shared__ __align__(16) unsigned char smem[];
    struct {
        int band_rows, max_w;
        const float* pose;
        vuda_frame fr;
    } a{band_rows, max_w, pose, fr};
    const int e = b.cam_env[cam];
    const int W = b.cam_w[cam], H = b.cam_h[cam];
    Band bd;
    bd.W = W;
    bd.y0 = y0;
    bd.y1 = min(H, bd.y0 + a.band_rows);
    bd.count = nullptr;

    unsigned char* p = smem;
    bd.z = reinterpret_cast<unsigned long long*>(p); p += (size_t)a.band_rows * a.max_w * 8;
    Bins bn;
    bn.rec = reinterpret_cast<BigRec*>(p); p += sizeof(BigRec) * kBigCap;
    int* vX = reinterpret_cast<int*>(p); p += 4 * kVcap;
    int* vY = reinterpret_cast<int*>(p); p += 4 * kVcap;
    float* viz = reinterpret_cast<float*>(p); p += 4 * kVcap;
    int* vflag = reinterpret_cast<int*>(p); p += 4 * kVcap;
    bn.tiles_x = (W + kTile - 1) / kTile;
    bn.ntiles = tiles_for(bd.y1 - bd.y0, W);
    const int ntiles_max = tiles_for(a.band_rows, a.max_w);
    bn.mask = reinterpret_cast<unsigned*>(p); p += 4 * (size_t)ntiles_max * kMaskWords;
    bn.nrec = reinterpret_cast<int*>(p); p += 4;
    unsigned* sflags = reinterpret_cast<unsigned*>(p); p += 12;

    const CamView cv = load_cam(b, cam);
    const int b0 = b.body_off[e];
    uint32_t* colors = b.tri_color + b.env_tri_base[e];

    if (threadIdx.x == 0) { *bn.nrec = 0; *sflags = 0u; }
    for (int i = threadIdx.x; i < bn.ntiles * kMaskWords; i += kRT) bn.mask[i] = 0u;
    init_band(bd);

    for (int ck = b.chunk_off[e]; ck < b.chunk_off[e + 1]; ck++) {
        const int cb0 = b.chunk_lo[ck];   // env-local first body, -1 = ground
        const int nv = b.chunk_nv[ck], nt = b.chunk_nt[ck];
        const int2* vt = b.vtab + b.chunk_vtab[ck];
        const uint2* tt = b.ttab + b.chunk_ttab[ck];
        const uint32_t tri0 = (uint32_t)b.chunk_tri0[ck];
        __syncthreads();  // the previous chunk's triangles are done with the vertex cache
        // 1. vertices
        for (int v = threadIdx.x; v < nv; v += kRT) {
            int X = 0, Y = 0;
            float iz = 0.0f;
            vflag[v] = project_vertex(b, a.pose, cv, b0, cb0, vt[v], X, Y, iz);
            vX[v] = X;
            vY[v] = Y;
            viz[v] = iz;
        }
        __syncthreads();
        // 2. triangles: strided over the CTA, no barrier until all are submitted
        for (int t = threadIdx.x; t < nt; t += kRT) {
            uint2 tv = tt[t];
            int i0 = tv.x & 0xffff, i1 = tv.x >> 16, i2 = tv.y;
            int fl = vflag[i0] | vflag[i1] | vflag[i2];
            if (fl == 0) {
                int X[3] = {vX[i0], vX[i1], vX[i2]};
                int Y[3] = {vY[i0], vY[i1], vY[i2]};
                float iz[3] = {viz[i0], viz[i1], viz[i2]};
                Tri tri;
                if (setup_tri(X, Y, iz, tri0 + (uint32_t)t, bd, tri)) submit_tri(tri, bd, bn);
            } else {
                // before the near plane or beyond the guard band: cull, clip or flag
                ClipFan f;
                const int cf = clip_near_fan(b, a.pose, cv, b0, cb0, vt[i0], vt[i1], vt[i2], f);
                if (cf) atomicOr(sflags, (unsigned)cf);
                for (int k = 0; k < f.n; k++) {
                    Tri tri;
                    if (setup_tri(f.X[k], f.Y[k], f.iz[k], tri0 + (uint32_t)t, bd, tri)) submit_tri(tri, bd, bn);
                }
            }
        }
        __syncthreads();
        // 3. binned triangles, tile by tile
        drain(bd, bn);
    }
    __syncthreads();

    // 4. resolve the band
    const int64_t pix0 = b.cam_pix_off[cam] + (int64_t)bd.y0 * W;
    const int npx = (bd.y1 - bd.y0) * W;
    uint8_t* rgb = a.fr.rgb + 3 * pix0;
    float* dep = a.fr.depth + pix0;
    uint32_t* tid = a.fr.triid ? a.fr.triid + pix0 : nullptr;
    const bool vec = ((pix0 & 3) == 0) && ((npx & 3) == 0);
    if (vec) {
        for (int q = threadIdx.x; q < (npx >> 2); q += kRT) {
            float d4[4];
            uint32_t t4[4];
            uint32_t c4[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                unsigned long long key = bd.z[4 * q + j];
                if (key == ~0ULL) {
                    d4[j] = 0.0f; t4[j] = 0xFFFFFFFFu; c4[j] = 0u;
                } else {
                    t4[j] = (uint32_t)(key & 0xFFFFFFFFull);
                    d4[j] = __uint_as_float((uint32_t)(key >> 32));
                    c4[j] = colors[t4[j]];
                }
            }
            reinterpret_cast<float4*>(dep)[q] = make_float4(d4[0], d4[1], d4[2], d4[3]);
            if (tid) reinterpret_cast<uint4*>(tid)[q] = make_uint4(t4[0], t4[1], t4[2], t4[3]);
            // 4 pixels = 12 bytes = 3 words, little endian r g b r | g b r g | b r g b
            uint32_t w0 = (c4[0] & 0xFFFFFFu) | ((c4[1] & 0xFFu) << 24);
            uint32_t w1 = ((c4[1] >> 8) & 0xFFFFu) | ((c4[2] & 0xFFFFu) << 16);
            uint32_t w2 = ((c4[2] >> 16) & 0xFFu) | ((c4[3] & 0xFFFFFFu) << 8);
            uint32_t* r32 = reinterpret_cast<uint32_t*>(rgb) + 3 * q;
            r32[0] = w0; r32[1] = w1; r32[2] = w2;
        }
    } else {
        for (int i = threadIdx.x; i < npx; i += kRT) {
            unsigned long long key = bd.z[i];
            uint32_t c = 0u;
            if (key == ~0ULL) {
                dep[i] = 0.0f;
                if (tid) tid[i] = 0xFFFFFFFFu;
            } else {
                uint32_t t = (uint32_t)(key & 0xFFFFFFFFull);
                dep[i] = __uint_as_float((uint32_t)(key >> 32));
                if (tid) tid[i] = t;
                c = colors[t];
            }
            rgb[3 * i] = c & 255u;
            rgb[3 * i + 1] = (c >> 8) & 255u;
            rgb[3 * i + 2] = (c >> 16) & 255u;
        }
    }
    if (threadIdx.x == 0 && *sflags) atomicOr(b.flags + e, *sflags);
}

__device__ __forceinline__ void load_desc(DevBatch& dst, const DevBatch& src) {
    const int* a = reinterpret_cast<const int*>(&src);
    int* d = reinterpret_cast<int*>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(DevBatch) / 4); k += blockDim.x) d[k] = a[k];
}

// Single batch: CTA i renders work item i of the batch.
__global__ void __launch_bounds__(kRT, 4) render_kernel(RenderArgs args) {
    __shared__ DevBatch sb;
    load_desc(sb, args.b);
    __syncthreads();
    render_band(sb, args.item_cam[blockIdx.x], args.item_y0[blockIdx.x], args.pose, args.fr, args.band_rows,
                args.max_w);
}

// Work list over several batches: persistent CTAs pull (batch, camera, band,
// pose slot) items from an atomic counter; frames come from each batch.
__global__ void __launch_bounds__(kRT, 4) render_list_kernel(const DevBatch* __restrict__ descs,
                                                             const int4* __restrict__ items, int nitems,
                                                             int* counter, int band_rows, int max_w, vuda_frame fr0,
                                                             int use_fr0, SmGate gate) {
    __shared__ DevBatch sb;
    __shared__ int s_item, s_gate;
    if (threadIdx.x == 0) s_gate = sm_gate_take(gate);
    __syncthreads();
    if (s_gate == kGateFull) return;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= nitems) break;
        const int4 it = items[item];
        load_desc(sb, descs[it.x & kItemDescMask]);
        __syncthreads();
        render_band(sb, it.y, it.z, sb.pose[(it.x >> 24) & 1], use_fr0 ? fr0 : sb.frame, band_rows, max_w);
        __syncthreads();
    }
    if (threadIdx.x == 0) sm_gate_release(gate, s_gate);
}

// Test hook: screen-space triangles, one CTA per band of the W x H image,
// through the same submit / tile-pass path as render_kernel.
__global__ void __launch_bounds__(kRT) raster_screen_kernel(const int32_t* __restrict__ xy,
                                                            const float* __restrict__ z, int ntri, int W, int H,
                                                            int band_rows, uint32_t* triid, float* depth,
                                                            uint32_t* count) {
    extern __shared__ __align__(16) unsigned char smem[];
    Band bd;
    bd.W = W;
    bd.y0 = blockIdx.x * band_rows;
    bd.y1 = min(H, bd.y0 + band_rows);
    unsigned char* p = smem;
    bd.z = reinterpret_cast<unsigned long long*>(p); p += (size_t)band_rows * W * 8;
    unsigned* scount = reinterpret_cast<unsigned*>(p); p += (size_t)band_rows * W * 4;
    Bins bn;
    bn.rec = reinterpret_cast<BigRec*>(p); p += sizeof(BigRec) * kBigCap;
    bn.tiles_x = (W + kTile - 1) / kTile;
    bn.ntiles = tiles_for(bd.y1 - bd.y0, W);
    bn.mask = reinterpret_cast<unsigned*>(p); p += 4 * (size_t)tiles_for(band_rows, W) * kMaskWords;
    bn.nrec = reinterpret_cast<int*>(p);
    bd.count = count ? scount : nullptr;
    if (threadIdx.x == 0) *bn.nrec = 0;
    for (int i = threadIdx.x; i < bn.ntiles * kMaskWords; i += kRT) bn.mask[i] = 0u;
    init_band(bd);
    __syncthreads();
    for (int t0 = 0; t0 < ntri; t0 += kBigCap) {   // at most kBigCap submissions between drains
        for (int t = t0 + threadIdx.x; t < min(ntri, t0 + kBigCap); t += kRT) {
            int X[3], Y[3];
            float iz[3];
#pragma unroll
            for (int v = 0; v < 3; v++) {
                X[v] = xy[6 * t + 2 * v];
                Y[v] = xy[6 * t + 2 * v + 1];
                iz[v] = 1.0f / z[3 * t + v];
            }
            // vertices beyond the guard band are discarded, as in the renderer
            bool out = false;
#pragma unroll
            for (int v = 0; v < 3; v++)
                out |= X[v] > kScreenLimit || X[v] < -kScreenLimit || Y[v] > kScreenLimit || Y[v] < -kScreenLimit;
            Tri tri;
            if (!out && setup_tri(X, Y, iz, (uint32_t)t, bd, tri)) submit_tri(tri, bd, bn);
        }
        __syncthreads();
        drain(bd, bn);
    }
    __syncthreads();
    int npx = (bd.y1 - bd.y0) * W;
    int64_t o = (int64_t)bd.y0 * W;
    for (int i = threadIdx.x; i < npx; i += kRT) {
        unsigned long long key = bd.z[i];
        if (key == ~0ULL) {
            triid[o + i] = 0xFFFFFFFFu;
            depth[o + i] = 0.0f;
        } else {
            triid[o + i] = (uint32_t)(key & 0xFFFFFFFFull);
            depth[o + i] = __uint_as_float((uint32_t)(key >> 32));
        }
        if (count) count[o + i] = scount[i];
    }
}

// Flat colour of every triangle of one unit from its world face normal
// (independent of the camera, so computed once per step for all cameras), by
// one warp.  Units [0, B) are bodies, [B, B + E) the ground quads.
__device__ __forceinline__ void shade_unit(const DevBatch& b, int unit, const float* __restrict__ pose) {
    const int lane = threadIdx.x & 31;
    const int B = b.B;
    int m;
    uint32_t alb;
    uint32_t* out;
    float R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    float s0 = 1, s1 = 1, s2 = 1, p0 = 0, p1 = 0, p2 = 0;
    bool body = unit < B;
    if (body) {
        const int g = unit;
        m = b.mesh_id[g];
        alb = b.albedo[g];
        out = b.tri_color + b.body_tri_base[g];
        quat_mat(pose[3 * B + g], pose[4 * B + g], pose[5 * B + g], pose[6 * B + g], R);
        s0 = b.scale[g]; s1 = b.scale[B + g]; s2 = b.scale[2 * B + g];
        p0 = pose[g]; p1 = pose[B + g]; p2 = pose[2 * B + g];
    } else {
        m = b.ground_mesh;
        alb = b.ground_albedo;
        out = b.tri_color + b.env_tri_base[unit - B];
    }
    const int t0 = b.mesh_tri_off[m], nt = b.mesh_tri_off[m + 1] - t0;
    const float* mv = b.mesh_verts + 3 * (size_t)b.mesh_vert_off[m];
    for (int t = lane; t < nt; t += 32) {
        const int32_t* tv = b.mesh_tris + 3 * (size_t)(t0 + t);
        float w[3][3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float* v = mv + 3 * tv[k];
            if (body) {
                float sx = s0 * v[0], sy = s1 * v[1], sz = s2 * v[2];
                float tx = (R[0] * sx + R[1] * sy) + R[2] * sz;
                float ty = (R[3] * sx + R[4] * sy) + R[5] * sz;
                float tz = (R[6] * sx + R[7] * sy) + R[8] * sz;
                w[k][0] = tx + p0; w[k][1] = ty + p1; w[k][2] = tz + p2;
            } else {
                w[k][0] = v[0]; w[k][1] = v[1]; w[k][2] = v[2];
            }
        }
        out[t] = flat_color(w[0], w[1], w[2], alb, b.light);
    }
}

__global__ void __launch_bounds__(256) shade_kernel(DevBatch b, const float* __restrict__ pose) {
    const int unit = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (unit >= b.B + b.E) return;
    shade_unit(b, unit, pose);
}

// Work list over several batches: warp w shades item w.
__global__ void __launch_bounds__(256) shade_list_kernel(const DevBatch* __restrict__ descs,
                                                         const int2* __restrict__ items, int nitems) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nitems) return;
    const int2 it = items[w];
    const DevBatch& b = descs[it.x & kItemDescMask];
    shade_unit(b, it.y, b.pose[(it.x >> 24) & 1]);
}

size_t screen_smem_bytes(int band_rows, int W) {
    int nt = tiles_for(band_rows, W);
    size_t s = (size_t)band_rows * W * 12 + sizeof(BigRec) * kBigCap + (size_t)nt * kMaskWords * 4 + 16;
    return (s + 15) & ~(size_t)15;
}

}  // namespace

cudaError_t launch_shade(const DevBatch& b, const float* pose, cudaStream_t stream) {
    if (b.B + b.E == 0) return cudaSuccess;
    const int units = b.B + b.E;
    shade_kernel<<<(units * 32 + 255) / 256, 256, 0, stream>>>(b, pose);
    return cudaGetLastError();
}

int render_vcap() { return kVcap; }
int render_chunk_bodies() { return kChunkBodies; }
size_t render_smem_for(int band_rows, int W) { return render_smem_bytes(band_rows, W); }

int render_default_band_rows(int max_w, int max_h) {
    // z-buffer of at most 32 KB per work item, in whole tiles
    int rows = 4096 / max_w;
    rows = rows >= kTile ? rows / kTile * kTile : (rows < 1 ? 1 : rows);
    return rows > max_h ? max_h : rows;
}

cudaError_t launch_render_items(const DevBatch& b, const float* pose, const vuda_frame& fr, const int32_t* item_cam,
                                const int32_t* item_y0, int nitems, int band_rows, int max_w, cudaStream_t stream) {
    if (nitems == 0) return cudaSuccess;
    size_t smem = render_smem_bytes(band_rows, max_w);
    // set on every launch: the attribute is tracked per context and the
    // kernel may be launched into different (green) contexts
    cudaError_t err = cudaFuncSetAttribute(render_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    err = launch_shade(b, pose, stream);
    if (err != cudaSuccess) return err;
    RenderArgs a;
    a.b = b;
    a.pose = pose;
    a.fr = fr;
    a.item_cam = item_cam;
    a.item_y0 = item_y0;
    a.band_rows = band_rows;
    a.max_w = max_w;
    render_kernel<<<nitems, kRT, smem, stream>>>(a);
    return cudaGetLastError();
}

int render_ctas_per_sm(int band_rows, int max_w) {
    int n = 0;
    size_t smem = render_smem_bytes(band_rows, max_w);
    cudaFuncSetAttribute(render_list_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, render_list_kernel, kRT, smem) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

CtaFootprint render_list_footprint(int band_rows, int max_w) {
    cudaFuncAttributes fa{};
    const int dyn = (int)render_smem_bytes(band_rows, max_w);
    if (cudaFuncGetAttributes(&fa, render_list_kernel) != cudaSuccess) return CtaFootprint{kRT, 255, 227 * 1024};
    return CtaFootprint{kRT, fa.numRegs, (int)fa.sharedSizeBytes + dyn};
}

cudaError_t launch_render_list(const DevBatch* descs, const int4* items, int nitems, int* counter, int grid,
                               const int2* shade_items, int nshade, int band_rows, int max_w, const vuda_frame* fr0,
                               SmGate gate, cudaStream_t stream) {
    cudaError_t err;
    if (nshade > 0) {
        shade_list_kernel<<<(nshade * 32 + 255) / 256, 256, 0, stream>>>(descs, shade_items, nshade);
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    if (nitems == 0) return cudaSuccess;
    size_t smem = render_smem_bytes(band_rows, max_w);
    err = cudaFuncSetAttribute(render_list_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(counter, 0, sizeof(int), stream);
    if (err != cudaSuccess) return err;
    vuda_frame f{};
    if (fr0) f = *fr0;
    render_list_kernel<<<grid, kRT, smem, stream>>>(descs, items, nitems, counter, band_rows, max_w, f, fr0 ? 1 : 0,
                                                    gate);
    return cudaGetLastError();
}

cudaError_t launch_raster_screen(const int32_t* xy, const float* z, int ntri, int W, int H, uint32_t* triid,
                                 float* depth, uint32_t* count, cudaStream_t stream) {
    int band_rows = 4096 / W;
    if (band_rows < 1) band_rows = 1;
    if (band_rows > H) band_rows = H;
    size_t smem = screen_smem_bytes(band_rows, W);
    cudaError_t err =
        cudaFuncSetAttribute(raster_screen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int grid = (H + band_rows - 1) / band_rows;
    raster_screen_kernel<<<grid, kRT, smem, stream>>>(xy, z, ntri, W, H, band_rows, triid, depth, count);
    return cudaGetLastError();
}

}  // namespace vuda
