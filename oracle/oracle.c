/* CPU oracle for the simulate-then-render step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this file's library; the product path
 * (the CUDA library and its binding) never does.  It shares no code with the
 * CUDA path: the only common inputs are the arrays of the seeded scene
 * generator.
 *
 * Plain, slow and sequential on purpose: one environment at a time, one
 * triangle at a time over its full bounding box into a full-frame z-buffer,
 * no tiling, binning or fusion.  Build: gcc -O2 -ffp-contract=off (no
 * fast-math), so every float expression is evaluated exactly in the written
 * order.
 *
 * What it computes (the paper fixes only the structure: a physics phase of
 * collision detection and constraint solving followed by a rendering phase
 * of vertex shading, rasterisation and fragment shading, Sec. 2.1; the
 * simulate/render dependency that lets sim(k+1) overlap render(k) is
 * Sec. 3.1):
 *   oracle_sim_step_f32 / _f64   physics step (physics.inc)
 *   oracle_contacts_f32          contact list of one environment
 *   oracle_render                per-environment camera render
 *   oracle_raster_screen_tris    rasteriser on given fixed-point triangles
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double dt;
    int substeps, iterations;
    double gravity[3];
    double restitution, restitution_threshold, friction, baumgarte, slop, margin, jacobi_omega;
    int plane, max_contacts_per_body;
    int gyroscopic;     /* 1: gyroscopic term of boxes (physics.inc) */
    int edge_contacts;  /* 1: box-box edge-edge contacts (physics.inc) */
    int hull_contacts;  /* 1: hulls collide through their vertices and faces (physics.inc) */
    /* meshes of the hull bodies (read only with hull_contacts) */
    const int* mesh_id;        /* mesh of each body: [B] for oracle_sim_step, [n] for oracle_contacts */
    const int* mesh_vert_off;  /* [M+1] */
    const float* mesh_verts;   /* [V][3] unit-size vertices */
    const int* mesh_tri_off;   /* [M+1] */
    const int* mesh_tris;      /* [T][3] vertex indices local to the mesh */
} oracle_params;

#define REAL float
#define FN(x) x##_f32
#define SQRT sqrtf
#define FABS fabsf
#include "physics.inc"
#undef REAL
#undef FN
#undef SQRT
#undef FABS

#define REAL double
#define FN(x) x##_f64
#define SQRT sqrt
#define FABS fabs
#include "physics.inc"
#undef REAL
#undef FN
#undef SQRT
#undef FABS

/* ------------------------------------------------------------------------ */
/* Rasteriser                                                                */
/* ------------------------------------------------------------------------ */
#define FLAG_GUARD 4u
#define SUBPIX 256.0f      /* 8 sub-pixel bits: fixed point 24.8 */
#define GUARD 16384.0f     /* |sx|, |sy| limit in pixels */
#define SCREEN_LIMIT 4194304 /* GUARD * SUBPIX: largest |X|, |Y| a snapped vertex can have */
#define NEAR_Z 0.01f

typedef struct {
    int ok;        /* 0: before the near plane or beyond the guard band */
    int X, Y;      /* snapped screen position, 24.8 fixed point */
    float iz;      /* 1 / view depth */
    float w[3];    /* world position */
    float v[3];    /* view position (xc, yc, zc) */
    unsigned flag; /* FLAG_GUARD, or 0 */
} overt;

/* Rasterise one triangle with snapped vertices (X[i], Y[i]) and inverse
 * depths iz[i] into a W x H z-buffer of 64-bit keys depth_bits << 32 | id.
 * The triangle is drawn iff it is counter-clockwise as seen by the camera
 * (negative signed area in y-down pixel coordinates).  count (optional)
 * receives one increment per covered pixel. */
static void raster_tri(const int* X, const int* Y, const float* izv, uint32_t id, int W, int H,
                       uint64_t* zbuf, int* count) {
    int64_t x0 = X[0], y0 = Y[0], x1 = X[1], y1 = Y[1], x2 = X[2], y2 = Y[2];
    int64_t area2 = (x1 - x0) * (y2 - y0) - (y1 - y0) * (x2 - x0);
    if (area2 >= 0) return;  /* back-facing or degenerate */
    /* reorder to positive area: vertices (0, 2, 1) */
    int64_t vx[3] = { x0, x2, x1 }, vy[3] = { y0, y2, y1 };
    float iz[3] = { izv[0], izv[2], izv[1] };
    area2 = -area2;
    int64_t A[3], B[3], C[3];
    int tl[3];
    for (int i = 0; i < 3; i++) {
        int j = (i + 1) % 3, k = (i + 2) % 3;
        A[i] = vy[j] - vy[k];
        B[i] = vx[k] - vx[j];
        C[i] = -A[i] * vx[j] - B[i] * vy[j];
        tl[i] = (A[i] > 0) || (A[i] == 0 && B[i] > 0);
    }
    /* pixel bounding box: centres 256 x + 128 inside [min, max] */
    int64_t mnx = vx[0], mxx = vx[0], mny = vy[0], mxy = vy[0];
    for (int i = 1; i < 3; i++) {
        if (vx[i] < mnx) mnx = vx[i];
        if (vx[i] > mxx) mxx = vx[i];
        if (vy[i] < mny) mny = vy[i];
        if (vy[i] > mxy) mxy = vy[i];
    }
    /* smallest x with 256 x + 128 >= mnx, largest with 256 x + 128 <= mxx */
    int64_t px0 = (mnx - 128 + 255) >> 8, px1 = (mxx - 128) >> 8;
    int64_t py0 = (mny - 128 + 255) >> 8, py1 = (mxy - 128) >> 8;
    if (px0 < 0) px0 = 0;
    if (py0 < 0) py0 = 0;
    if (px1 > W - 1) px1 = W - 1;
    if (py1 > H - 1) py1 = H - 1;
    float af = (float)area2;
    for (int64_t py = py0; py <= py1; py++) {
        for (int64_t px = px0; px <= px1; px++) {
            int64_t cx = 256 * px + 128, cy = 256 * py + 128;
            int64_t E[3];
            int in = 1;
            for (int i = 0; i < 3; i++) {
                E[i] = A[i] * cx + B[i] * cy + C[i];
                if (!(E[i] > 0 || (E[i] == 0 && tl[i]))) in = 0;
            }
            if (!in) continue;
            float den = ((float)E[0] * iz[0] + (float)E[1] * iz[1]) + (float)E[2] * iz[2];
            float depth = af / den;
            uint32_t bits;
            memcpy(&bits, &depth, 4);
            uint64_t key = ((uint64_t)bits << 32) | id;
            uint64_t* z = zbuf + py * W + px;
            if (key < *z) *z = key;
            if (count) count[py * W + px]++;
        }
    }
}

/* Rasterise ntri screen-space triangles given as snapped 24.8 fixed-point
 * vertices xy[t][v][2] and view depths z[t][v] into W x H buffers of the
 * nearest triangle id (0xFFFFFFFF where empty) and its depth (0 where empty).
 * count (optional) gets the number of triangles covering each pixel.  As in
 * the renderer, a triangle with a vertex beyond the 2^14-pixel guard band
 * (|x| or |y| above 2^22 in 1/256 px) is discarded. */
int oracle_raster_screen_tris(const int32_t* xy, const float* z, int ntri, int W, int H,
                              uint32_t* triid, float* depth, int* count) {
    if (W <= 0 || H <= 0 || ntri < 0) return 1;
    uint64_t* zb = malloc(sizeof(uint64_t) * (size_t)W * H);
    for (size_t i = 0; i < (size_t)W * H; i++) zb[i] = ~(uint64_t)0;
    if (count) memset(count, 0, sizeof(int) * (size_t)W * H);
    for (int t = 0; t < ntri; t++) {
        int X[3], Y[3];
        float iz[3];
        for (int v = 0; v < 3; v++) {
            X[v] = xy[6 * t + 2 * v];
            Y[v] = xy[6 * t + 2 * v + 1];
            iz[v] = 1.0f / z[3 * t + v];
        }
        int out = 0;
        for (int v = 0; v < 3; v++)
            if (X[v] > SCREEN_LIMIT || X[v] < -SCREEN_LIMIT || Y[v] > SCREEN_LIMIT || Y[v] < -SCREEN_LIMIT) out = 1;
        if (out) continue;
        raster_tri(X, Y, iz, (uint32_t)t, W, H, zb, count);
    }
    for (size_t i = 0; i < (size_t)W * H; i++) {
        if (zb[i] == ~(uint64_t)0) {
            triid[i] = 0xFFFFFFFFu;
            depth[i] = 0.0f;
        } else {
            triid[i] = (uint32_t)(zb[i] & 0xFFFFFFFFu);
            uint32_t bits = (uint32_t)(zb[i] >> 32);
            memcpy(depth + i, &bits, 4);
        }
    }
    free(zb);
    return 0;
}

/* world position of mesh vertex v under pose (p, q) and per-axis scale s */
static void transform_vertex(const float* v, const float* s, const float* p, const float* q, float* w) {
    float R[9];
    quat_to_mat_f32(q, R);
    float sv[3] = { s[0] * v[0], s[1] * v[1], s[2] * v[2] };
    float t[3];
    mat_vec_f32(R, sv, t);
    w[0] = t[0] + p[0];
    w[1] = t[1] + p[1];
    w[2] = t[2] + p[2];
}

/* Snapped screen position of a view-space point with zc >= near: sx = W/2 +
 * fpy xc / zc, sy = H/2 - fpy yc / zc, rounded to 1/256 px (half to even).
 * Returns 0, or FLAG_GUARD if the point lies beyond the guard band. */
static unsigned snap_view(float xc, float yc, float zc, float fpy, int W, int H, int* X, int* Y, float* iz) {
    float sx = (float)W * 0.5f + (fpy * xc) / zc;
    float sy = (float)H * 0.5f - (fpy * yc) / zc;
    if (!(fabsf(sx) < GUARD && fabsf(sy) < GUARD)) return FLAG_GUARD;
    *X = (int)rintf(sx * SUBPIX);
    *Y = (int)rintf(sy * SUBPIX);
    *iz = 1.0f / zc;
    return 0;
}

static void project_vertex(overt* o, const float* eye, const float* rt, const float* up, const float* fw,
                           float fpy, int W, int H) {
    float d[3] = { o->w[0] - eye[0], o->w[1] - eye[1], o->w[2] - eye[2] };
    o->v[0] = (rt[0] * d[0] + rt[1] * d[1]) + rt[2] * d[2];
    o->v[1] = (up[0] * d[0] + up[1] * d[1]) + up[2] * d[2];
    o->v[2] = (fw[0] * d[0] + fw[1] * d[1]) + fw[2] * d[2];
    o->ok = 0;
    o->flag = 0;
    if (!(o->v[2] >= NEAR_Z)) return;   /* before the near plane: its triangles are clipped */
    o->flag = snap_view(o->v[0], o->v[1], o->v[2], fpy, W, H, &o->X, &o->Y, &o->iz);
    o->ok = o->flag == 0;
}

/* 1 if all three vertices lie beyond the same side plane of the view
 * frustum -- right of the image (fpy xc > W/2 zc, i.e. sx > W in front of
 * the camera), left (fpy xc < -W/2 zc), above (fpy yc > H/2 zc) or below
 * (fpy yc < -H/2 zc).  Each plane passes through the eye, so the triangle
 * lies in that half-space and covers no pixel, wherever its vertices are
 * (also behind the camera). */
static int outside_frustum_side(const overt* const* tv, float fpy, int W, int H) {
    const float hw = (float)W * 0.5f, hh = (float)H * 0.5f;
    int r = 1, l = 1, u = 1, d = 1;
    for (int i = 0; i < 3; i++) {
        const float* v = tv[i]->v;
        r &= fpy * v[0] > hw * v[2];
        l &= fpy * v[0] < -(hw * v[2]);
        u &= fpy * v[1] > hh * v[2];
        d &= fpy * v[1] < -(hh * v[2]);
    }
    return r | l | u | d;
}

/* Sutherland-Hodgman clipping of triangle (a, b, c) against the near plane
 * zc = NEAR_Z, keeping the part with zc >= NEAR_Z.  The clipped polygon (3
 * or 4 vertices, in the triangle's order) is cut into a fan from its first
 * vertex; each triangle of the fan is rasterised with the original
 * triangle's id.  A new vertex on an edge from an inside vertex p to an
 * outside vertex q is p + t (q - p) with t = (near - p_z) / (q_z - p_z),
 * always taken from the inside end, so that the two triangles sharing the
 * edge get the same point; it lies on the plane (zc = near exactly).
 * Returns FLAG_GUARD (and draws nothing) if a vertex of the polygon lies
 * beyond the guard band, else 0.  (With every vertex in front of the plane
 * the polygon is the triangle itself.) */
static unsigned clip_near_and_raster(const overt* const* tv, uint32_t id, float fpy, int W, int H, uint64_t* zb) {
    int X[4], Y[4];
    float iz[4];
    int n = 0;
    for (int i = 0; i < 3; i++) {
        const overt* p = tv[i];
        const overt* q = tv[(i + 1) % 3];
        const int pin = p->v[2] >= NEAR_Z, qin = q->v[2] >= NEAR_Z;
        if (pin) {
            if (p->flag) return p->flag;
            X[n] = p->X; Y[n] = p->Y; iz[n] = p->iz;
            n++;
        }
        if (pin != qin) {
            const overt* a = pin ? p : q;   /* inside end */
            const overt* b = pin ? q : p;   /* outside end */
            float t = (NEAR_Z - a->v[2]) / (b->v[2] - a->v[2]);
            float xc = a->v[0] + t * (b->v[0] - a->v[0]);
            float yc = a->v[1] + t * (b->v[1] - a->v[1]);
            unsigned f = snap_view(xc, yc, NEAR_Z, fpy, W, H, X + n, Y + n, iz + n);
            if (f) return f;
            n++;
        }
    }
    for (int k = 1; k + 1 < n; k++) {
        int fx[3] = { X[0], X[k], X[k + 1] }, fy[3] = { Y[0], Y[k], Y[k + 1] };
        float fz[3] = { iz[0], iz[k], iz[k + 1] };
        raster_tri(fx, fy, fz, id, W, H, zb, NULL);
    }
    return 0;
}

/* flat colour of a triangle from its world-space face normal */
static uint32_t shade(const float* w0, const float* w1, const float* w2, uint32_t albedo, const float* L) {
    float e1[3] = { w1[0] - w0[0], w1[1] - w0[1], w1[2] - w0[2] };
    float e2[3] = { w2[0] - w0[0], w2[1] - w0[1], w2[2] - w0[2] };
    float n[3];
    cross3_f32(e1, e2, n);
    float len = sqrtf(dot3_f32(n, n));
    float ndl = 0.0f;
    if (len > 0.0f) {
        float u[3] = { n[0] / len, n[1] / len, n[2] / len };
        ndl = dot3_f32(u, L);
    }
    float I = 0.2f + 0.8f * (ndl > 0.0f ? ndl : 0.0f);
    uint32_t out = 0;
    for (int c = 0; c < 3; c++) {
        float a = (float)((albedo >> (8 * c)) & 255u);
        int v = (int)(a * I + 0.5f);
        if (v > 255) v = 255;
        out |= (uint32_t)v << (8 * c);
    }
    return out;
}

/* Render every camera of every environment.  Poses are SoA planes pos[3][B],
 * quat[4][B].  Outputs are concatenated per camera (cam_pix_off[c] is the
 * first pixel of camera c): rgb[px][3] u8, depth[px] f32 (view depth, 0 for
 * background), triid[px] u32 (env-local id, 0xFFFFFFFF for background).
 * Triangle ids: the ground mesh's triangles first, then body b's triangles
 * in the order of the environment's bodies and of each mesh. */
int oracle_render(int num_envs, const int32_t* body_off, int B, const float* pos, const float* quat,
                  const int32_t* mesh_id, const float* mesh_scale, const uint32_t* albedo,
                  const int32_t* mesh_vert_off, const float* mesh_verts,
                  const int32_t* mesh_tri_off, const int32_t* mesh_tris,
                  int ground_mesh, uint32_t ground_albedo,
                  const int32_t* cam_off, const int32_t* cam_w, const int32_t* cam_h,
                  const float* cam_eye, const float* cam_right, const float* cam_up, const float* cam_fwd,
                  const float* cam_fpy, const float* light, const int64_t* cam_pix_off,
                  uint8_t* rgb, float* depth, uint32_t* triid, uint32_t* env_flags) {
    for (int e = 0; e < num_envs; e++) {
        int b0 = body_off[e], nb = body_off[e + 1] - b0;
        for (int c = cam_off[e]; c < cam_off[e + 1]; c++) {
            int W = cam_w[c], H = cam_h[c];
            const float *eye = cam_eye + 3 * c, *rt = cam_right + 3 * c, *up = cam_up + 3 * c,
                        *fw = cam_fwd + 3 * c;
            float fpy = cam_fpy[c];
            size_t npx = (size_t)W * H;
            uint64_t* zb = malloc(sizeof(uint64_t) * npx);
            for (size_t i = 0; i < npx; i++) zb[i] = ~(uint64_t)0;
            /* colour table for this environment, indexed by triangle id */
            int ntri = mesh_tri_off[ground_mesh + 1] - mesh_tri_off[ground_mesh];
            for (int b = 0; b < nb; b++) {
                int m = mesh_id[b0 + b];
                ntri += mesh_tri_off[m + 1] - mesh_tri_off[m];
            }
            uint32_t* color = malloc(sizeof(uint32_t) * (size_t)(ntri > 0 ? ntri : 1));
            uint32_t id = 0;
            for (int b = -1; b < nb; b++) {
                int m = b < 0 ? ground_mesh : mesh_id[b0 + b];
                int v0 = mesh_vert_off[m], nv = mesh_vert_off[m + 1] - v0;
                overt* vs = malloc(sizeof(overt) * (size_t)(nv > 0 ? nv : 1));
                float p[3], q[4], s[3];
                uint32_t alb = ground_albedo;
                if (b >= 0) {
                    int g = b0 + b;
                    for (int k = 0; k < 3; k++) { p[k] = pos[k * B + g]; s[k] = mesh_scale[k * B + g]; }
                    for (int k = 0; k < 4; k++) q[k] = quat[k * B + g];
                    alb = albedo[g];
                }
                for (int v = 0; v < nv; v++) {
                    const float* mv = mesh_verts + 3 * (v0 + v);
                    if (b < 0) { vs[v].w[0] = mv[0]; vs[v].w[1] = mv[1]; vs[v].w[2] = mv[2]; }
                    else transform_vertex(mv, s, p, q, vs[v].w);
                    project_vertex(vs + v, eye, rt, up, fw, fpy, W, H);
                }
                for (int t = mesh_tri_off[m]; t < mesh_tri_off[m + 1]; t++, id++) {
                    const int32_t* tv = mesh_tris + 3 * t;
                    const overt *a = vs + tv[0], *bb = vs + tv[1], *cc = vs + tv[2];
                    color[id] = shade(a->w, bb->w, cc->w, alb, light);
                    if (!a->ok || !bb->ok || !cc->ok) {
                        /* a vertex before the near plane or beyond the guard
                         * band: nothing to draw if the triangle lies wholly
                         * before the near plane or beyond one image edge;
                         * else clip it (which flags a guard-band vertex) */
                        const overt* tvs[3] = { a, bb, cc };
                        const int nin = (a->v[2] >= NEAR_Z) + (bb->v[2] >= NEAR_Z) + (cc->v[2] >= NEAR_Z);
                        if (nin == 0 || outside_frustum_side(tvs, fpy, W, H)) continue;
                        env_flags[e] |= clip_near_and_raster(tvs, id, fpy, W, H, zb);
                        continue;
                    }
                    int X[3] = { a->X, bb->X, cc->X }, Y[3] = { a->Y, bb->Y, cc->Y };
                    float iz[3] = { a->iz, bb->iz, cc->iz };
                    raster_tri(X, Y, iz, id, W, H, zb, NULL);
                }
                free(vs);
            }
            int64_t o = cam_pix_off[c];
            for (size_t i = 0; i < npx; i++) {
                uint8_t* px = rgb + 3 * (o + (int64_t)i);
                if (zb[i] == ~(uint64_t)0) {
                    px[0] = px[1] = px[2] = 0;
                    depth[o + i] = 0.0f;
                    if (triid) triid[o + i] = 0xFFFFFFFFu;
                } else {
                    uint32_t t = (uint32_t)(zb[i] & 0xFFFFFFFFu);
                    uint32_t bits = (uint32_t)(zb[i] >> 32);
                    memcpy(depth + o + i, &bits, 4);
                    if (triid) triid[o + i] = t;
                    uint32_t col = color[t];
                    px[0] = col & 255u; px[1] = (col >> 8) & 255u; px[2] = (col >> 16) & 255u;
                }
            }
            free(color);
            free(zb);
        }
    }
    return 0;
}
