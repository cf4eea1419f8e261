// Face planes of the mesh library for hull contacts: one thread per
// triangle, evaluated once when a batch is created.  The expressions are
// written in the order that defines them (the library is built without FMA
// contraction, with IEEE division and square root), so every plane is the
// correctly rounded evaluation of the same formula wherever it is used.
// Also the mesh vertices padded to 16 bytes (one load per vertex in the
// face searches).
#include <cuda_runtime.h>

#include <cmath>

#include "internal.cuh"

namespace vuda {
namespace {

__global__ void mesh_planes_kernel(const float* __restrict__ verts, const int32_t* __restrict__ vert_off,
                                   const int32_t* __restrict__ tri_off, const int32_t* __restrict__ tris, int M,
                                   int T, float4* __restrict__ planes) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    int lo = 0, hi = M - 1;   // the mesh of triangle t: the last whose first triangle is <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tri_off[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const int v0 = vert_off[lo];
    float u[3][3];
#pragma unroll
    for (int q = 0; q < 3; q++)
#pragma unroll
        for (int c = 0; c < 3; c++) u[q][c] = verts[3 * (v0 + tris[3 * t + q]) + c];
    const float e1x = u[1][0] - u[0][0], e1y = u[1][1] - u[0][1], e1z = u[1][2] - u[0][2];
    const float e2x = u[2][0] - u[0][0], e2y = u[2][1] - u[0][1], e2z = u[2][2] - u[0][2];
    const float cx = e1y * e2z - e1z * e2y;
    const float cy = e1z * e2x - e1x * e2z;
    const float cz = e1x * e2y - e1y * e2x;
    const float len = sqrtf((cx * cx + cy * cy) + cz * cz);
    if (len > 0.0f) {
        const float nx = cx / len, ny = cy / len, nz = cz / len;
        planes[t] = make_float4(nx, ny, nz, (nx * u[0][0] + ny * u[0][1]) + nz * u[0][2]);
    } else {
        planes[t] = make_float4(0.0f, 0.0f, 0.0f, INFINITY);   // no plane: every depth below it is -inf
    }
}

__global__ void mesh_vert4_kernel(const float* __restrict__ verts, int V, float4* __restrict__ vert4) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V) vert4[v] = make_float4(verts[3 * v], verts[3 * v + 1], verts[3 * v + 2], 0.0f);
}

}  // namespace

cudaError_t launch_mesh_planes(const float* verts, const int32_t* vert_off, const int32_t* tri_off,
                               const int32_t* tris, int num_meshes, int num_tris, float4* planes, int num_verts,
                               float4* vert4, cudaStream_t stream) {
    if (num_verts > 0)
        mesh_vert4_kernel<<<(num_verts + 127) / 128, 128, 0, stream>>>(verts, num_verts, vert4);
    if (num_tris > 0 && num_meshes > 0)
        mesh_planes_kernel<<<(num_tris + 127) / 128, 128, 0, stream>>>(verts, vert_off, tri_off, tris, num_meshes,
                                                                        num_tris, planes);
    return cudaGetLastError();
}

}  // namespace vuda
