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
constexpr float kNear = 0.01f;          // view depth below which a vertex invalidates its triangles
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
// quad): world = R(q) (s * v) + p, view = basis . (world - eye), projected
// and snapped to 24.8 fixed point.  Returns 0 and sets X, Y, iz, or returns
// the discard flag (near plane or guard band); the world position is set
// either way.
__device__ __forceinline__ int project_vertex(const DevBatch& b, const float* __restrict__ pose, const CamView& c,
                                              int b0, int cb0, int2 ent, int& X, int& Y, float& iz, float& wx,
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
    float xc = (c.rx * dx + c.ry * dy) + c.rz * dz;
    float yc = (c.ux * dx + c.uy * dy) + c.uz * dz;
    float zc = (c.fx * dx + c.fy * dy) + c.fz * dz;
    if (!(zc >= kNear)) return VUDA_FLAG_NEAR_DISCARD;
    float sxp = c.hw + (c.fpy * xc) / zc;
    float syp = c.hh - (c.fpy * yc) / zc;
    if (!(fabsf(sxp) < kGuard && fabsf(syp) < kGuard)) return VUDA_FLAG_GUARD_DISCARD;
    X = __float2int_rn(sxp * 256.0f);
    Y = __float2int_rn(syp * 256.0f);
    iz = 1.0f / zc;
    return 0;
}

__device__ __forceinline__ int project_vertex(const DevBatch& b, const float* __restrict__ pose, const CamView& c,
                                              int b0, int cb0, int2 ent, int& X, int& Y, float& iz) {
    float wx, wy, wz;
    return project_vertex(b, pose, c, b0, cb0, ent, X, Y, iz, wx, wy, wz);
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
