// Pooled observation of a rendered frame (vuda_observe): for a policy that
// acts between steps on what the renderer produced.  One CTA per camera;
// each thread sums the pixels of cells (row by row) and writes the cell's
// mean view depth (scaled) and mean luminance.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace vuda {
namespace {

__global__ void observe_kernel(const uint8_t* __restrict__ rgb, const float* __restrict__ depth,
                               const int64_t* __restrict__ cam_pix_off, const int32_t* __restrict__ cam_w,
                               const int32_t* __restrict__ cam_h, int cams_per_env, int cells, float depth_scale,
                               float* __restrict__ out) {
    const int cam = blockIdx.x;
    const int e = cam / cams_per_env, cl = cam % cams_per_env;
    const int W = cam_w[cam], H = cam_h[cam];
    const int cw = W / cells, ch = H / cells;
    const int64_t p0 = cam_pix_off[cam];
    const int ncell = cells * cells;
    const int64_t row = (int64_t)2 * cams_per_env * ncell;   // floats per environment
    const float L0 = 0.299f / 255.0f, L1 = 0.587f / 255.0f, L2 = 0.114f / 255.0f;
    const float inv = 1.0f / (float)(cw * ch);
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        const int cy = c / cells, cx = c % cells;
        float sd = 0.0f, sl = 0.0f;
        for (int y = 0; y < ch; y++) {
            const int64_t p = p0 + (int64_t)(cy * ch + y) * W + (int64_t)cx * cw;
            for (int x = 0; x < cw; x++) {
                sd = sd + __ldg(depth + p + x);
                const uint8_t* q = rgb + 3 * (p + x);
                sl = sl + (((float)__ldg(q) * L0 + (float)__ldg(q + 1) * L1) + (float)__ldg(q + 2) * L2);
            }
        }
        out[e * row + (int64_t)cl * ncell + c] = (sd * inv) * depth_scale;
        out[e * row + (int64_t)(cams_per_env + cl) * ncell + c] = sl * inv;
    }
}

}  // namespace

cudaError_t launch_observe(const DevBatch& b, const vuda_frame& fr, int cams_per_env, int cells, float depth_scale,
                           float* out, cudaStream_t stream) {
    if (b.C == 0) return cudaSuccess;
    const int threads = cells * cells < 256 ? ((cells * cells + 31) / 32) * 32 : 256;
    observe_kernel<<<b.C, threads, 0, stream>>>(fr.rgb, fr.depth, b.cam_pix_off, b.cam_w, b.cam_h, cams_per_env,
                                                cells, depth_scale, out);
    return cudaGetLastError();
}

}  // namespace vuda
