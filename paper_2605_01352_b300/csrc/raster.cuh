// Device helpers shared by the two render paths (band kernel in render.cu,
// tiled kernels in tiled.cu): constants of the fixed-point pipeline, the
// vertex transform and projection, the exact int64 -> float conversion.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace vuda {

constexpr int kTile = 16;               // tile edge in pixels
constexpr int kVertexCache = 1024;      // vertices of one chunk of bodies (shared-memory vertex cache)
constexpr float kNear = 0.01f;          // near plane: triangles are clipped to view depth >= kNear
constexpr int kVertBehind = 0x100;      // project_vertex: the vertex lies before the near plane (not a status bit)
constexpr float kGuard = 16384.0f;      // |sx|, |sy| limit of the guard band, pixels
constexpr int kScreenLimit = 4194304;   // kGuard x 256: largest |X|, |Y| of a snapped vertex

__device__ __forceinline__ void quat_mat(float w, float x, float y, float z, float* R) {
    R[0] = 1.0f - 2.0f * (y * y + z * z);
    R[1] = 2.0f * (x * y - w * z);
    R[2] = 2.0f * (x * z + w * y);
    R[3] = 2.0f * (x * y + w * z);
    R[4] = 1.0f - 2.0f * (x * x + z * z);
    R[5] = 2.0f * (y * z - w * x);
    R[6] = 2.0f * (x * z - w * y);
    R[7] = 2.0f * (y * z + w * x);
    R[8] = 1.0f - 2.0f * (x * x + y * y);
}

// int64 -> float, round to nearest even, without the 64-bit conversion
// (which runs on the narrow FP64 pipe).  Split x = H 2^23 + R with
// H = floor(x / 2^23) and 0 <= R < 2^23.  For |x| <= 2^47 (every edge value
// and doubled area inside the guard band) |H| <= 2^24, so H 2^23 and R are
// both exact floats, their exact sum is x, and one IEEE single-precision
// addition returns RN(x): the same value as the correctly rounded
// conversion.  R goes through the exponent-bias identity
// float(2^23 + R) - 2^23 = R (exact for R < 2^23).
__device__ __forceinline__ float i64_to_f32(long long x) {
    const int H = (int)(x >> 23);
    const unsigned R = (unsigned)x & 0x7FFFFFu;
    const float hf = __int2float_rn(H) * 8388608.0f;
    const float rf = __uint_as_float(0x4B000000u | R) - 8388608.0f;
    return hf + rf;
}

// Camera of one view: eye, right / up / forward basis, focal length in
// pixels, image centre.
struct CamView {
    float ex, ey, ez, rx, ry, rz, ux, uy, uz, fx, fy, fz, fpy, hw, hh;
};

__device__ __forceinline__ CamView load_cam(const DevBatch& b, int cam) {
    const float* cp = b.cam_par + (size_t)cam * kCamWords;
    CamView c;
    c.ex = cp[0]; c.ey = cp[1]; c.ez = cp[2];
    c.rx = cp[3]; c.ry = cp[4]; c.rz = cp[5];
    c.ux = cp[6]; c.uy = cp[7]; c.uz = cp[8];
    c.fx = cp[9]; c.fy = cp[10]; c.fz = cp[11];
    c.fpy = cp[12];
    c.hw = (float)b.cam_w[cam] * 0.5f;
    c.hh = (float)b.cam_h[cam] * 0.5f;
    return c;
}

// Vertex ent of a chunk whose first env-local body is cb0 (-1 = the ground
// quad): world = R(q) (s * v) + p and view = basis . (world - eye).
__device__ __forceinline__ void view_vertex(const DevBatch& b, const float* __restrict__ pose, const CamView& c,
                                            int b0, int cb0, int2 ent, float& xc, float& yc, float& zc, float& wx,
                                            float& wy, float& wz) {
    const int B = b.B;
    const int bi = cb0 + ent.y;
    const float* mv = b.mesh_verts + 3 * (size_t)ent.x;
    if (bi < 0) {
        wx = mv[0]; wy = mv[1]; wz = mv[2];
    } else {
        const int g = b0 + bi;
        float R[9];
        quat_mat(pose[3 * B + g], pose[4 * B + g], pose[5 * B + g], pose[6 * B + g], R);
        float sx = b.scale[g] * mv[0], sy = b.scale[B + g] * mv[1], sz = b.scale[2 * B + g] * mv[2];
        float tx = (R[0] * sx + R[1] * sy) + R[2] * sz;
        float ty = (R[3] * sx + R[4] * sy) + R[5] * sz;
        float tz = (R[6] * sx + R[7] * sy) + R[8] * sz;
        wx = tx + pose[g];
        wy = ty + pose[B + g];
        wz = tz + pose[2 * B + g];
    }
    float dx = wx - c.ex, dy = wy - c.ey, dz = wz - c.ez;
    xc = (c.rx * dx + c.ry * dy) + c.rz * dz;
    yc = (c.ux * dx + c.uy * dy) + c.uz * dz;
    zc = (c.fx * dx + c.fy * dy) + c.fz * dz;
}

// Snapped screen position of a view-space point with zc >= kNear:
// sx = W/2 + fpy xc / zc, sy = H/2 - fpy yc / zc, rounded to 24.8 fixed
// point (half to even).  Returns 0, or VUDA_FLAG_GUARD_DISCARD beyond the
// guard band.
__device__ __forceinline__ int snap_view(const CamView& c, float xc, float yc, float zc, int& X, int& Y, float& iz) {
    float sxp = c.hw + (c.fpy * xc) / zc;
    float syp = c.hh - (c.fpy * yc) / zc;
    if (!(fabsf(sxp) < kGuard && fabsf(syp) < kGuard)) return VUDA_FLAG_GUARD_DISCARD;
    X = __float2int_rn(sxp * 256.0f);
    Y = __float2int_rn(syp * 256.0f);
    iz = 1.0f / zc;
    return 0;
}

// Projected vertex: returns 0 and sets X, Y, iz; kVertBehind before the
// near plane (its triangles are clipped); or VUDA_FLAG_GUARD_DISCARD.  The
// world position is set in every case.
__device__ __forceinline__ int project_vertex(const DevBatch& b, const float* __restrict__ pose, const CamView& c,
                                              int b0, int cb0, int2 ent, int& X, int& Y, float& iz, float& wx,
                                              float& wy, float& wz) {
    float xc, yc, zc;
    view_vertex(b, pose, c, b0, cb0, ent, xc, yc, zc, wx, wy, wz);
    if (!(zc >= kNear)) return kVertBehind;
    return snap_view(c, xc, yc, zc, X, Y, iz);
}

__device__ __forceinline__ int project_vertex(const DevBatch& b, const float* __restrict__ pose, const CamView& c,
                                              int b0, int cb0, int2 ent, int& X, int& Y, float& iz) {
    float wx, wy, wz;
    return project_vertex(b, pose, c, b0, cb0, ent, X, Y, iz, wx, wy, wz);
}

// Sutherland-Hodgman clipping of a triangle (view-space vertices v[0..2], at
// least one of them before the near plane) against zc = kNear, keeping the
// part with zc >= kNear, cut into a fan from the clipped polygon's first
// vertex.  A new vertex on an edge from an inside vertex a to an outside
// vertex b is a + t (b - a), t = (near - a.z) / (b.z - a.z), always taken
// from the inside end so that both triangles sharing the edge get the same
// point, and lies on the plane.  Writes n (0, 1 or 2) fan triangles as
// snapped vertices in the triangle's order; returns
// VUDA_FLAG_GUARD_DISCARD (and n = 0) if a polygon vertex lies beyond the
// guard band.
__device__ __forceinline__ int clip_near(const float (&v)[3][3], const CamView& c, int (&X)[2][3], int (&Y)[2][3],
                                         float (&iz)[2][3], int& n) {
    int PX[4], PY[4];
    float PZ[4];
    int np = 0;
    n = 0;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int j = i == 2 ? 0 : i + 1;
        const bool pin = v[i][2] >= kNear, qin = v[j][2] >= kNear;
        if (pin) {
            if (snap_view(c, v[i][0], v[i][1], v[i][2], PX[np], PY[np], PZ[np])) return VUDA_FLAG_GUARD_DISCARD;
            np++;
        }
        if (pin != qin) {
            const int ia = pin ? i : j, ib = pin ? j : i;
            const float t = (kNear - v[ia][2]) / (v[ib][2] - v[ia][2]);
            const float xc = v[ia][0] + t * (v[ib][0] - v[ia][0]);
            const float yc = v[ia][1] + t * (v[ib][1] - v[ia][1]);
            if (snap_view(c, xc, yc, kNear, PX[np], PY[np], PZ[np])) return VUDA_FLAG_GUARD_DISCARD;
            np++;
        }
    }
    for (int k = 1; k + 1 < np; k++, n++) {
        X[n][0] = PX[0]; X[n][1] = PX[k]; X[n][2] = PX[k + 1];
        Y[n][0] = PY[0]; Y[n][1] = PY[k]; Y[n][2] = PY[k + 1];
        iz[n][0] = PZ[0]; iz[n][1] = PZ[k]; iz[n][2] = PZ[k + 1];
    }
    return 0;
}

// True if all three view-space vertices lie beyond the same side plane of
// the view frustum: right of the image (fpy xc > W/2 zc), left
// (fpy xc < -W/2 zc), above (fpy yc > H/2 zc) or below (fpy yc < -H/2 zc).
// Each plane passes through the eye, so such a triangle covers no pixel,
// wherever its vertices are (also behind the camera).
__device__ __forceinline__ bool outside_frustum_side(const float (&v)[3][3], const CamView& c) {
    bool r = true, l = true, u = true, d = true;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        r = r && (c.fpy * v[i][0] > c.hw * v[i][2]);
        l = l && (c.fpy * v[i][0] < -(c.hw * v[i][2]));
        u = u && (c.fpy * v[i][1] > c.hh * v[i][2]);
        d = d && (c.fpy * v[i][1] < -(c.hh * v[i][2]));
    }
    return r || l || u || d;
}

// The fan triangles of a clipped triangle.
struct ClipFan {
    int X[2][3], Y[2][3];
    float iz[2][3];
    int n;
};

// A triangle with chunk vertices e0, e1, e2 of which at least one lies
// before the near plane or beyond the guard band: their view positions are
// recomputed exactly as project_vertex computed them; nothing is drawn if
// the triangle lies wholly before the near plane or beyond one side plane
// of the frustum; otherwise it is clipped (a guard-band vertex in front of
// the plane discards it with the flag).  Out of line: the path is rare and
// must not add registers to the callers' triangle loops.  Returns 0 or
// VUDA_FLAG_GUARD_DISCARD.
static __device__ __noinline__ int clip_near_fan(const DevBatch& b, const float* __restrict__ pose, const CamView& c,
                                                 int b0, int cb0, int2 e0, int2 e1, int2 e2, ClipFan& f) {
    float v[3][3], wx, wy, wz;
    view_vertex(b, pose, c, b0, cb0, e0, v[0][0], v[0][1], v[0][2], wx, wy, wz);
    view_vertex(b, pose, c, b0, cb0, e1, v[1][0], v[1][1], v[1][2], wx, wy, wz);
    view_vertex(b, pose, c, b0, cb0, e2, v[2][0], v[2][1], v[2][2], wx, wy, wz);
    f.n = 0;
    if (!(v[0][2] >= kNear) && !(v[1][2] >= kNear) && !(v[2][2] >= kNear)) return 0;
    if (outside_frustum_side(v, c)) return 0;
    return clip_near(v, c, f.X, f.Y, f.iz, f.n);
}

// Flat colour of a triangle with world vertices w0, w1, w2 (mesh order):
// I = 0.2 + 0.8 max(0, n . L) with n the normalised face normal
// (w1 - w0) x (w2 - w0), each 8-bit channel of the albedo scaled by I,
// rounded and clamped.
__device__ __forceinline__ uint32_t flat_color(const float* w0, const float* w1, const float* w2, uint32_t alb,
                                               const float* light) {
    float e1x = w1[0] - w0[0], e1y = w1[1] - w0[1], e1z = w1[2] - w0[2];
    float e2x = w2[0] - w0[0], e2y = w2[1] - w0[1], e2z = w2[2] - w0[2];
    float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
    float len = sqrtf((nx * nx + ny * ny) + nz * nz);
    float ndl = 0.0f;
    if (len > 0.0f) ndl = ((nx / len) * light[0] + (ny / len) * light[1]) + (nz / len) * light[2];
    float I = 0.2f + 0.8f * (ndl > 0.0f ? ndl : 0.0f);
    uint32_t col = 0;
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        float av = (float)((alb >> (8 * ch)) & 255u);
        int vv = (int)(av * I + 0.5f);
        vv = vv > 255 ? 255 : vv;
        col |= (uint32_t)vv << (8 * ch);
    }
    return col;
}

}  // namespace vuda
