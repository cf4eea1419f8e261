// Batched rigid-body step (the physics phase of the simulate-then-render
// loop; the paper characterises it as collision detection plus constraint
// solving in many fine-grained, low-occupancy stages, Sec. 2.1).
//
// One CTA of VUDA_SIM_THREADS threads owns one environment for a whole
// launch: its bodies and contacts live in shared memory across all
// substeps, so the serial chain of substeps x (contacts + Jacobi iterations)
// runs on block barriers instead of kernel launches.  This file is compiled
// twice: 128 threads per environment (physics.cu, namespace vuda) for the
// common case of a few dozen bodies, and 512 threads (physics_wide.cu,
// namespace vuda::wide) for environments of more than 64 bodies.
//
// Arithmetic: every float expression is evaluated in the written order
// (the library is built with -fmad=false), so results reproduce a plain
// sequential evaluation of the same formulas.
//
// Per substep (h = dt / substeps):
//   1. v += h (g + F / m); rotation R(q) and world inverse inertia R I^-1 R^T
//   2. contacts in canonical order: plane contacts by body (box corners in
//      sign-bit order), then pairs (i, j), i < j, that pass a bounding-sphere
//      test: sphere-sphere, sphere-box, box-box (A's corners inside B, then
//      B's corners inside A); capacity max_contacts_per_body * N
//   3. per contact: lever arms, tangent basis, mass-split effective masses,
//      velocity target (speculative for d >= 0, bias beyond slop, restitution)
//   4. Jacobi iterations: every contact solves against the iteration's
//      velocities, then every body sums its contacts' impulses in ascending
//      contact order
//   5. x += h v, q <- normalize(q + h/2 (0, w) q)
#pragma once
#ifndef VUDA_SIM_THREADS
#error "define VUDA_SIM_THREADS (threads per environment) before including physics_impl.cuh"
#endif
#include <cuda_runtime.h>

#include "internal.cuh"

namespace vuda {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Field indices of a contact record (kContactWords floats in eight 16-byte
// groups: n|KN, rA|VMIN, rB|LN, t1|KT1, t2|KT2, P|LT1, LA|LT2, LB|AB).
// KN, KT1, KT2 hold the effective masses k; P is the impulse of the
// current iteration, LA = rA x P and LB = rB x P its angular parts.  Between
// generation and the per-contact constants, RA holds the contact point and
// VMIN the distance.
enum : int {
    F_N = 0, F_KN = 3, F_RA = 4, F_VMIN = 7, F_RB = 8, F_LN = 11, F_T1 = 12, F_KT1 = 15, F_T2 = 16, F_KT2 = 19,
    F_P = 20, F_LT1 = 23, F_LA = 24, F_LT2 = 27, F_LB = 28, F_AB = 31
};
static_assert(F_AB + 1 == kContactWords, "contact record layout");

// One contact record: kContactWords fields at p[0..), records kCS words apart.
constexpr int kCS = kContactStride;
struct Rec {
    float* p;
    __device__ __forceinline__ float& operator[](int f) const { return p[f]; }
    // the 16-byte group starting at field f (a multiple of 4)
    __device__ __forceinline__ float4& g(int f) const { return *reinterpret_cast<float4*>(p + f); }
};

struct Contacts {
    float* s;       // shared records [cap][kCS]
    int cap;        // records in shared memory
    float* g;       // global spill records (record c at c - cap)
    __device__ __forceinline__ Rec rec(int c) const {
        return c < cap ? Rec{s + c * kCS} : Rec{g + (size_t)(c - cap) * kCS};
    }
};

// The same records when all of them are in shared memory.
struct SmemContacts {
    float* s;
    __device__ __forceinline__ Rec rec(int c) const { return Rec{s + c * kCS}; }
};

// Per-env bodies in shared memory: one record of kBW words per body.  The
// odd stride keeps 32 consecutive bodies on 32 different banks, and every
// field sits at an immediate offset from the record base.
enum : int {
    B_P = 0, B_Q = 3, B_V = 7, B_W = 10, B_D = 13, B_IM = 16, B_II = 17, B_BR = 20, B_R = 21, B_I = 30,
    B_TYPE = 39, B_NCB = 40
};
constexpr int kBW = 41;

struct Bodies {
    float* base;
    int* loff;
    __device__ __forceinline__ float* b(int i) const { return base + i * kBW; }
    __device__ __forceinline__ float& P(int k, int i) const { return b(i)[B_P + k]; }
    __device__ __forceinline__ float& Q(int k, int i) const { return b(i)[B_Q + k]; }
    __device__ __forceinline__ float& V(int k, int i) const { return b(i)[B_V + k]; }
    __device__ __forceinline__ float& W(int k, int i) const { return b(i)[B_W + k]; }
    __device__ __forceinline__ float& D(int k, int i) const { return b(i)[B_D + k]; }
    __device__ __forceinline__ float& Rm(int k, int i) const { return b(i)[B_R + k]; }
    __device__ __forceinline__ float& I(int k, int i) const { return b(i)[B_I + k]; }
    __device__ __forceinline__ float& IM(int i) const { return b(i)[B_IM]; }
    __device__ __forceinline__ float& II(int k, int i) const { return b(i)[B_II + k]; }
    __device__ __forceinline__ float& BR(int i) const { return b(i)[B_BR]; }
    __device__ __forceinline__ int& TYPE(int i) const { return reinterpret_cast<int*>(b(i))[B_TYPE]; }
    __device__ __forceinline__ int& NCB(int i) const { return reinterpret_cast<int*>(b(i))[B_NCB]; }
};

struct f3 { float x, y, z; };

__device__ __forceinline__ float dot3(f3 a, f3 b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
__device__ __forceinline__ f3 cross3(f3 a, f3 b) {
    return f3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ f3 sub3(f3 a, f3 b) { return f3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 add3(f3 a, f3 b) { return f3{a.x + b.x, a.y + b.y, a.z + b.z}; }

__device__ __forceinline__ f3 ldpos(const Bodies& B, int i) { return f3{B.P(0, i), B.P(1, i), B.P(2, i)}; }
__device__ __forceinline__ f3 ldvel(const Bodies& B, int i) { return f3{B.V(0, i), B.V(1, i), B.V(2, i)}; }
__device__ __forceinline__ f3 ldang(const Bodies& B, int i) { return f3{B.W(0, i), B.W(1, i), B.W(2, i)}; }

// R v with R row major in the body's 9 planes
__device__ __forceinline__ f3 rmul(const Bodies& B, int i, f3 v) {
    return f3{(B.Rm(0, i) * v.x + B.Rm(1, i) * v.y) + B.Rm(2, i) * v.z,
              (B.Rm(3, i) * v.x + B.Rm(4, i) * v.y) + B.Rm(5, i) * v.z,
              (B.Rm(6, i) * v.x + B.Rm(7, i) * v.y) + B.Rm(8, i) * v.z};
}
// R^T v
__device__ __forceinline__ f3 rtmul(const Bodies& B, int i, f3 v) {
    return f3{(B.Rm(0, i) * v.x + B.Rm(3, i) * v.y) + B.Rm(6, i) * v.z,
              (B.Rm(1, i) * v.x + B.Rm(4, i) * v.y) + B.Rm(7, i) * v.z,
              (B.Rm(2, i) * v.x + B.Rm(5, i) * v.y) + B.Rm(8, i) * v.z};
}
// Iw v
__device__ __forceinline__ f3 imul(const Bodies& B, int i, f3 v) {
    return f3{(B.I(0, i) * v.x + B.I(1, i) * v.y) + B.I(2, i) * v.z,
              (B.I(3, i) * v.x + B.I(4, i) * v.y) + B.I(5, i) * v.z,
              (B.I(6, i) * v.x + B.I(7, i) * v.y) + B.I(8, i) * v.z};
}

__device__ __forceinline__ f3 box_corner(const Bodies& B, int i, int k) {
    f3 l{(k & 1) ? B.D(0, i) : -B.D(0, i), (k & 2) ? B.D(1, i) : -B.D(1, i), (k & 4) ? B.D(2, i) : -B.D(2, i)};
    f3 w = rmul(B, i, l);
    return add3(w, ldpos(B, i));
}

__device__ __forceinline__ void put_contact(const Contacts& C, int c, int a, int b, f3 n, f3 p, float d) {
    Rec r = C.rec(c);
    r.g(F_N) = make_float4(n.x, n.y, n.z, 0.0f);
    r.g(F_RA) = make_float4(p.x, p.y, p.z, d);   // point and distance, converted later
    r.g(F_LB) = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(a | ((b + 1) << 16)));
}

// Sphere s against box x: normal from the box to the sphere, point on the box, distance.
__device__ __forceinline__ void sphere_box(const Bodies& B, int s, int x, f3& n, f3& pt, float& d) {
    f3 ps = ldpos(B, s), px = ldpos(B, x);
    float h[3] = {B.D(0, x), B.D(1, x), B.D(2, x)};
    float r = B.D(0, s);
    f3 l3 = rtmul(B, x, sub3(ps, px));
    float l[3] = {l3.x, l3.y, l3.z}, q[3], nl[3], pl[3];
#pragma unroll
    for (int k = 0; k < 3; k++) q[k] = l[k] < -h[k] ? -h[k] : (l[k] > h[k] ? h[k] : l[k]);
    if (q[0] != l[0] || q[1] != l[1] || q[2] != l[2]) {
        f3 df{l[0] - q[0], l[1] - q[1], l[2] - q[2]};
        float dist = sqrtf(dot3(df, df));
        nl[0] = df.x / dist; nl[1] = df.y / dist; nl[2] = df.z / dist;
        d = dist - r;
        pl[0] = q[0]; pl[1] = q[1]; pl[2] = q[2];
    } else {
        float pen[3];
#pragma unroll
        for (int k = 0; k < 3; k++) pen[k] = h[k] - fabsf(l[k]);
        // axis of least penetration (lowest index on ties), selected without
        // indexing the arrays by it, so that they stay in registers
        const bool m1 = pen[1] < pen[0];
        const float pm01 = m1 ? pen[1] : pen[0];
        const bool m2 = pen[2] < pm01;
        const int m = m2 ? 2 : (m1 ? 1 : 0);
        const float penm = m2 ? pen[2] : pm01;
        const float lm = m2 ? l[2] : (m1 ? l[1] : l[0]);
        float sg = lm >= 0.0f ? 1.0f : -1.0f;
        d = -penm - r;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            nl[k] = k == m ? sg : 0.0f;
            pl[k] = k == m ? sg * h[k] : l[k];
        }
    }
    n = rmul(B, x, f3{nl[0], nl[1], nl[2]});
    pt = add3(rmul(B, x, f3{pl[0], pl[1], pl[2]}), px);
}

// Corner k of box a tested against box b: returns true if within the margin.
__device__ __forceinline__ bool corner_in_box(const Bodies& B, int a, int b, int k, float margin, f3& c, f3& nB,
                                              float& d) {
    c = box_corner(B, a, k);
    f3 l3 = rtmul(B, b, sub3(c, ldpos(B, b)));
    float l[3] = {l3.x, l3.y, l3.z};
    float pen[3];
#pragma unroll
    for (int j = 0; j < 3; j++) pen[j] = B.D(j, b) - fabsf(l[j]);
    // axis of least penetration (lowest index on ties), selected without
    // indexing the arrays by it
    const bool m1 = pen[1] < pen[0];
    const float pm01 = m1 ? pen[1] : pen[0];
    const bool m2 = pen[2] < pm01;
    const int m = m2 ? 2 : (m1 ? 1 : 0);
    d = -(m2 ? pen[2] : pm01);
    if (!(d < margin)) return false;
    const float lm = m2 ? l[2] : (m1 ? l[1] : l[0]);
    float sg = lm >= 0.0f ? 1.0f : -1.0f;
    nB = f3{sg * B.Rm(m, b), sg * B.Rm(3 + m, b), sg * B.Rm(6 + m, b)};  // column m of R_b
    return true;
}

__device__ __forceinline__ bool is_box(const Bodies& B, int i) { return B.TYPE(i) == kShapeBox; }

__device__ __forceinline__ f3 rcol(const Bodies& B, int i, int k) { return f3{B.Rm(k, i), B.Rm(3 + k, i), B.Rm(6 + k, i)}; }

// Edge-edge contact of boxes a (the pair's A) and b (B): the separating-
// axis test of two oriented boxes in the formulation of Gottschalk, Lin and
// Manocha (OBBTree, 1996), over C_kl = a_k . b_l, t = p_a - p_b, t_k = t . a_k
// and u_l = t . b_l: A's face k: |t_k| - (h_a,k + sum_m h_b,m |C_km|); B's
// face l: |u_l| - (sum_m h_a,m |C_ml| + h_b,l); edge a_k x b_l ((k, k1, k2),
// (l, l1, l2) cyclic): (|t_k2 C_k1,l - t_k1 C_k2,l| - (h_a,k1 |C_k2,l| +
// h_a,k2 |C_k1,l|) - (h_b,l1 |C_k,l2| + h_b,l2 |C_k,l1|)) / sqrt(1 - C_kl^2),
// edges with 1 - C_kl^2 <= 1e-6 skipped.  The greatest separation wins (the
// first on ties; an edge axis must beat the best so far by more than 1e-5 m,
// near ties with a face go to the face).  An edge axis with a separation
// below the margin gives one contact: normal +-(a_k x b_l) normalised, from B
// to A; distance the separation; point midway between the closest points of
// A's edge along a_k furthest towards B and B's edge along b_l furthest
// towards A (segment closest points: s clamped, t from s and clamped, then s
// from t and clamped if t was clamped).
// (kCopy: the kernel variant that uses it)
template <int kCopy>
__device__ __forceinline__ bool box_edge_edge(const Bodies& B, int a, int b, float margin, f3& nout, f3& pt,
                                           float& d) {
    const f3 dp = sub3(ldpos(B, a), ldpos(B, b));
    float Cm[3][3], AC[3][3], ta[3], tb[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        ta[k] = dot3(dp, rcol(B, a, k));
        tb[k] = dot3(dp, rcol(B, b, k));
#pragma unroll
        for (int l = 0; l < 3; l++) {
            Cm[k][l] = dot3(rcol(B, a, k), rcol(B, b, l));
            AC[k][l] = fabsf(Cm[k][l]);
        }
    }
    const float ha[3] = {B.D(0, a), B.D(1, a), B.D(2, a)};
    const float hb[3] = {B.D(0, b), B.D(1, b), B.D(2, b)};
    float best = 0.0f;
    int bq = -1;
    // a face axis separating the boxes by the margin or more decides the
    // test (the winning separation can only be larger): skip the edge axes
    float face = -3.0e38f;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        face = fmaxf(face, fabsf(ta[k]) - (ha[k] + ((hb[0] * AC[k][0] + hb[1] * AC[k][1]) + hb[2] * AC[k][2])));
        face = fmaxf(face, fabsf(tb[k]) - (((ha[0] * AC[0][k] + ha[1] * AC[1][k]) + ha[2] * AC[2][k]) + hb[k]));
    }
    if (!(face < margin)) return false;
#pragma unroll
    for (int q = 0; q < 15; q++) {
        float sep;
        if (q < 3) {
            const int k = q;
            sep = fabsf(ta[k]) - (ha[k] + ((hb[0] * AC[k][0] + hb[1] * AC[k][1]) + hb[2] * AC[k][2]));
        } else if (q < 6) {
            const int l = q - 3;
            sep = fabsf(tb[l]) - (((ha[0] * AC[0][l] + ha[1] * AC[1][l]) + ha[2] * AC[2][l]) + hb[l]);
        } else {
            const int k = (q - 6) / 3, l = (q - 6) % 3;
            const int k1 = (k + 1) % 3, k2 = (k + 2) % 3, l1 = (l + 1) % 3, l2 = (l + 2) % 3;
            const float len2 = 1.0f - Cm[k][l] * Cm[k][l];
            if (!(len2 > 1e-6f)) continue;
            const float tl = fabsf(ta[k2] * Cm[k1][l] - ta[k1] * Cm[k2][l]);
            const float ra = ha[k1] * AC[k2][l] + ha[k2] * AC[k1][l];
            const float rb = hb[l1] * AC[k][l2] + hb[l2] * AC[k][l1];
            sep = ((tl - ra) - rb) / sqrtf(len2);
        }
        if (bq < 0 || sep > best + (q < 6 ? 0.0f : 1e-5f)) {
            best = sep;
            bq = q;
        }
    }
    if (bq < 6 || !(best < margin)) return false;
    const int k = (bq - 6) / 3, l = (bq - 6) % 3;
    f3 bu;
    {
        const f3 c = cross3(rcol(B, a, k), rcol(B, b, l));
        const float len = sqrtf(dot3(c, c));
        bu = f3{c.x / len, c.y / len, c.z / len};
    }
    const float sg = dot3(dp, bu) >= 0.0f ? 1.0f : -1.0f;
    const f3 n{sg * bu.x, sg * bu.y, sg * bu.z};
    f3 cA = ldpos(B, a), cB = ldpos(B, b);
#pragma unroll
    for (int m = 0; m < 3; m++) {
        const f3 am = rcol(B, a, m), bm = rcol(B, b, m);
        if (m != k) {
            const float s1 = dot3(n, am) > 0.0f ? -B.D(m, a) : B.D(m, a);
            cA = f3{cA.x + s1 * am.x, cA.y + s1 * am.y, cA.z + s1 * am.z};
        }
        if (m != l) {
            const float s2 = dot3(n, bm) > 0.0f ? B.D(m, b) : -B.D(m, b);
            cB = f3{cB.x + s2 * bm.x, cB.y + s2 * bm.y, cB.z + s2 * bm.z};
        }
    }
    const f3 ea = rcol(B, a, k), eb = rcol(B, b, l);
    const f3 r = sub3(cA, cB);
    const float bb = dot3(ea, eb), cc = dot3(ea, r), ff = dot3(eb, r);
    const float den = 1.0f - bb * bb;
    const float hak = B.D(k, a), hbl = B.D(l, b);
    float sA = (bb * ff - cc) / den;
    sA = sA < -hak ? -hak : (sA > hak ? hak : sA);
    float tB = ff + sA * bb;
    if (tB < -hbl || tB > hbl) {
        tB = tB < -hbl ? -hbl : hbl;
        sA = tB * bb - cc;
        sA = sA < -hak ? -hak : (sA > hak ? hak : sA);
    }
    pt = f3{0.5f * ((cA.x + sA * ea.x) + (cB.x + tB * eb.x)), 0.5f * ((cA.y + sA * ea.y) + (cB.y + tB * eb.y)),
            0.5f * ((cA.z + sA * ea.z) + (cB.z + tB * eb.z))};
    nout = n;
    d = best;
    return true;
}

// Gyroscopic term of a box: the torque-free Euler equations I dw/dt =
// -w x I w in the body frame, one implicit step by one Newton iteration
// from the current angular velocity (E. Catto, "Numerical Methods", GDC
// 2015): f = h w x (I w), J = I + h (skew(w) I - skew(I w)), D = -J^-1 f
// (adjugate and determinant), and the world angular velocity gains R D.
__device__ __forceinline__ void gyroscopic(const Bodies& S, int i, const float* R, float ib0, float ib1, float ib2,
                                        float h) {
    const float wx = S.W(0, i), wy = S.W(1, i), wz = S.W(2, i);
    // w = R^T w_world
    const float w0 = (R[0] * wx + R[3] * wy) + R[6] * wz;
    const float w1 = (R[1] * wx + R[4] * wy) + R[7] * wz;
    const float w2 = (R[2] * wx + R[5] * wy) + R[8] * wz;
    const float I0 = 1.0f / ib0, I1 = 1.0f / ib1, I2 = 1.0f / ib2;
    const float L0 = I0 * w0, L1 = I1 * w1, L2 = I2 * w2;
    const float f0 = h * (w1 * L2 - w2 * L1), f1 = h * (w2 * L0 - w0 * L2), f2 = h * (w0 * L1 - w1 * L0);
    const float J00 = I0, J11 = I1, J22 = I2;
    const float J01 = h * (w2 * (I2 - I1)), J02 = h * (w1 * (I2 - I1));
    const float J10 = h * (w2 * (I0 - I2)), J12 = h * (w0 * (I0 - I2));
    const float J20 = h * (w1 * (I1 - I0)), J21 = h * (w0 * (I1 - I0));
    const float A00 = J11 * J22 - J12 * J21, A01 = J02 * J21 - J01 * J22, A02 = J01 * J12 - J02 * J11;
    const float A10 = J12 * J20 - J10 * J22, A11 = J00 * J22 - J02 * J20, A12 = J02 * J10 - J00 * J12;
    const float A20 = J10 * J21 - J11 * J20, A21 = J01 * J20 - J00 * J21, A22 = J00 * J11 - J01 * J10;
    const float det = (J00 * A00 + J01 * A10) + J02 * A20;
    const float D0 = -(((A00 * f0 + A01 * f1) + A02 * f2) / det);
    const float D1 = -(((A10 * f0 + A11 * f1) + A12 * f2) / det);
    const float D2 = -(((A20 * f0 + A21 * f1) + A22 * f2) / det);
    S.W(0, i) = wx + ((R[0] * D0 + R[1] * D1) + R[2] * D2);
    S.W(1, i) = wy + ((R[3] * D0 + R[4] * D1) + R[5] * D2);
    S.W(2, i) = wz + ((R[6] * D0 + R[7] * D1) + R[8] * D2);
}

constexpr int kT = VUDA_SIM_THREADS;   // threads per environment (one CTA)
constexpr int kParts = kT / 32;        // parts of the contact list, one per warp, when building per-body lists
constexpr int kMinCtas = kT == 128 ? 7 : 2;   // CTAs per SM the register budget is set for
constexpr int kPairChunk = 4 * kT;  // candidate pairs per round of the pair phase (4 per thread)

__device__ __forceinline__ bool broad(const Bodies& B, int i, int j, float margin) {
    f3 dx = sub3(ldpos(B, i), ldpos(B, j));
    float d2 = dot3(dx, dx);
    float rs = (B.BR(i) + B.BR(j)) + margin;
    return d2 < rs * rs;
}

// Edge tests of the box pairs among passing pairs [w0, w1), one thread
// each, into slots (2 float4 per pair: normal and distance, point and hit).
// Inlined, like the other optional passes: an out-of-line call makes the
// kernel keep values across it in local memory, which with seven CTAs'
// shared memory on the SM has little L1 left to hold it (measured slower).
template <int kCopy>
__device__ __forceinline__ void edge_prepass(const Bodies& S, const int* plist, int w0, int w1, float4* slots,
                                          float margin) {
    for (int q = w0 + (int)threadIdx.x; q < w1; q += kT) {
        const int pr = plist[q];
        const int i = pr & 0xffff, j = pr >> 16;
        if (!(is_box(S, i) && is_box(S, j))) continue;
        f3 n{0.0f, 0.0f, 0.0f}, pt{0.0f, 0.0f, 0.0f};
        float d = 0.0f;
        const bool h = box_edge_edge<kCopy>(S, i, j, margin, n, pt, d);
        slots[2 * (q - w0)] = make_float4(n.x, n.y, n.z, d);
        slots[2 * (q - w0) + 1] = make_float4(pt.x, pt.y, pt.z, h ? 1.0f : 0.0f);
    }
}

// One narrow-phase test of pair (i, j): sub 0 for sphere-sphere and
// sphere-box; for box-box sub 0..7 tests A's corner sub inside B and
// sub 8..15 tests B's corner sub-8 inside A (sub 16, the crossing edges,
// is computed before the item pass).
__device__ __forceinline__ bool pair_test(const Bodies& B, int i, int j, int sub, float margin, f3& n, f3& pt, float& d) {
    bool bi = is_box(B, i), bj = is_box(B, j);
    if (!bi && !bj) {
        f3 pa = ldpos(B, i), pb = ldpos(B, j);
        f3 dx = sub3(pa, pb);
        float d2 = dot3(dx, dx);
        float ra = B.D(0, i), rb = B.D(0, j);
        float dist = sqrtf(d2);
        if (dist > 0.0f) n = f3{dx.x / dist, dx.y / dist, dx.z / dist};
        else n = f3{0.0f, 0.0f, 1.0f};
        d = (dist - ra) - rb;
        pt = f3{pa.x - n.x * ra, pa.y - n.y * ra, pa.z - n.z * ra};
        return d < margin;
    }
    // one call site per test (the narrow phase is inlined): the box of a
    // sphere-box pair, or the box whose corner is tested, given explicitly;
    // the normal always points from j to i
    bool flip;
    bool hit;
    if (!bi || !bj) {
        flip = bi;   // box i, sphere j: the test gives the normal from i to j
        sphere_box(B, bi ? j : i, bi ? i : j, n, pt, d);
        hit = d < margin;
    } else {
        flip = sub >= 8;   // B's corner inside A: the normal from i to j
        hit = corner_in_box(B, flip ? j : i, flip ? i : j, sub & 7, margin, pt, n, d);
    }
    if (flip) n = f3{-n.x, -n.y, -n.z};
    return hit;
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Shared scratch of the CTA-wide scans: two halves of kT/32 ints used by
// consecutive scans in turn.  A scan needs one barrier (between the warps'
// writes and everyone's reads): a thread writes a half again only two scans
// later, after passing the barrier of the scan in between, which every
// reader of the half reaches only after its reads.
struct ScanBuf {
    int* w;     // [2][kT / 32]
    int k;      // scans so far (the same in every thread)
};

// Exclusive prefix sum over the CTA's kT threads in thread order.  Must be
// called by all threads, in the same sequence of scans.
__device__ __forceinline__ int block_excl_scan(int v, ScanBuf& sb, int& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int* wsum = sb.w + (sb.k & 1) * (kT / 32);
    sb.k++;
    int x = warp_incl_scan(v, lane);
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    int off = 0;
    total = 0;
#pragma unroll
    for (int k = 0; k < kT / 32; k++) {
        int s = wsum[k];
        if (k < w) off += s;
        total += s;
    }
    return off + x - v;
}

__device__ __forceinline__ void unpack_ab(const Rec& r, int& a, int& b) {
    int ab = __float_as_int(r.g(F_LB).w);   // a 128-bit load: no bank conflict across consecutive records
    a = ab & 0xffff;
    b = (ab >> 16) - 1;
}


// mass-split effective mass along dir
__device__ __forceinline__ float eff_mass(const Bodies& B, int a, int b, f3 rA, f3 rB, f3 dir) {
    f3 u = cross3(rA, dir);
    float kA = (float)B.NCB(a) * (B.IM(a) + dot3(u, imul(B, a, u)));
    float kB = 0.0f;
    if (b >= 0) {
        u = cross3(rB, dir);
        kB = (float)B.NCB(b) * (B.IM(b) + dot3(u, imul(B, b, u)));
    }
    return kA + kB;
}

__device__ __forceinline__ f3 rel_vel(const Bodies& B, int a, int b, f3 rA, f3 rB) {
    f3 va = add3(ldvel(B, a), cross3(ldang(B, a), rA));
    if (b >= 0) {
        f3 vb = add3(ldvel(B, b), cross3(ldang(B, b), rB));
        return sub3(va, vb);
    }
    return va;
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Bytes of per-env shared memory before the contact records.
__host__ __device__ inline size_t phys_fixed_bytes(int NB, int cmax) {
    size_t f = (size_t)kBW * NB * 4;         // body records
    f += (size_t)(NB + 1) * 4;               // loff[NB+1]
    f += (size_t)kParts * NB * 4;            // per-part list counters
    f += (size_t)kPairChunk * (4 + 2);       // passing pairs and their first item
    f += (size_t)2 * (kT / 32) * 4;          // scan scratch
    f += (size_t)8 * NB * 2;                 // plane items (u16: body << 3 | corner)
    f += (size_t)2 * cmax * 2;               // per-body contact lists (u16: contact << 1 | side)
    return align16(f);
}

// First pair (i, j), i < j, of flat index k in lexicographic order.
__device__ __forceinline__ void pair_of_index(int k, int N, int& i, int& j) {
    // start(i) = i (2N - i - 1) / 2 is the flat index of (i, i + 1)
    float b = (float)(2 * N - 1);
    float disc = b * b - 8.0f * (float)k;
    int ii = (int)floorf((b - sqrtf(fmaxf(disc, 0.0f))) * 0.5f);
    ii = max(0, min(ii, N - 2));
    auto start = [N](int x) { return x * (2 * N - x - 1) / 2; };
    while (ii > 0 && start(ii) > k) ii--;
    while (ii < N - 2 && start(ii + 1) <= k) ii++;
    i = ii;
    j = k - start(ii) + ii + 1;
}

// Ordered expansion over the CTA: each thread offers `nsub` sub-items for its
// unit; returns the exclusive item prefix and the total (block scan).
// Items are later tested one per thread and their hits compacted in order.

// One environment for nsteps steps, by the whole CTA.  b lives in shared
// memory (copied there by the kernels below).
// Per-body contact lists, per-contact constants and the Jacobi iterations of
// one substep.  CA is the contact-record accessor: shared memory only when
// every contact of the env fits there (the common case, 32-bit shared
// addressing), or shared then global spill.
template <class CA>
__device__ __forceinline__ void solve_substep(const CA& C, const Bodies& S, int* qcnt, unsigned short* lists,
                                              ScanBuf& wsum, int nc, int N, int NB, const SimConst& sc, float h) {
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    // contacts per body, and per-body lists (contact << 1 | side) in
    // ascending contact order: the list is cut into kParts parts, the
    // contacts of each body are counted per part (qcnt is zero on entry),
    // and warp q fills the entries of part q
    __syncthreads();   // the contact records of this substep are written
    const int qlen = (nc + kParts - 1) / kParts;
    for (int c = tid; c < nc; c += kT) {
        int a, bb;
        unpack_ab(C.rec(c), a, bb);
        int q;   // c / qlen (c < kParts qlen)
        if (kParts == 4) q = (c >= qlen) + (c >= 2 * qlen) + (c >= 3 * qlen);
        else q = c / qlen;
        atomicAdd(qcnt + q * NB + a, 1);
        if (bb >= 0) atomicAdd(qcnt + q * NB + bb, 1);
    }
    __syncthreads();
    // warp q fills the entries of the contacts of part q; every warp forms
    // the list offsets itself (a warp scan of the bodies' counts), so no CTA
    // barrier separates counting from filling; warp 0 keeps the counts and
    // offsets for the later phases
    {
        int run = 0;
        for (int i0 = 0; i0 < N; i0 += 32) {
            const int i = i0 + lane;
            int v = 0, before = 0;
            if (i < N) {
#pragma unroll
                for (int q = 0; q < kParts; q++) {
                    const int cq = qcnt[q * NB + i];
                    if (q < warp) before += cq;
                    v += cq;
                }
            }
            const int incl = warp_incl_scan(v, lane);
            const int lo = run + incl - v;
            run += __shfl_sync(kFull, incl, 31);
            if (i >= N) continue;
            if (warp == 0) {
                S.NCB(i) = v;
                S.loff[i] = lo;
            }
            int o = lo + before;
            int cend = min(nc, (warp + 1) * qlen);
            int c = warp * qlen;
            for (; c + 4 <= cend; c += 4) {
                int ab[4];
#pragma unroll
                for (int u = 0; u < 4; u++) ab[u] = __float_as_int(C.rec(c + u).g(F_LB).w);
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    int a = ab[u] & 0xffff, bb = (ab[u] >> 16) - 1;
                    if (a == i) lists[o++] = (unsigned short)((c + u) << 1);
                    else if (bb == i) lists[o++] = (unsigned short)(((c + u) << 1) | 1);
                }
            }
            for (; c < cend; c++) {
                int a, bb;
                unpack_ab(C.rec(c), a, bb);
                if (a == i) lists[o++] = (unsigned short)(c << 1);
                else if (bb == i) lists[o++] = (unsigned short)((c << 1) | 1);
            }
        }
        if (warp == 0 && lane == 0) S.loff[N] = run;
    }
    __syncthreads();

    // 3. per-contact constants
    for (int c = tid; c < nc; c += kT) {
        Rec r = C.rec(c);
        const float4 gn = r.g(F_N), gp = r.g(F_RA);
        const int ab = __float_as_int(r.g(F_LB).w);
        const int a = ab & 0xffff, bb = (ab >> 16) - 1;
        f3 n{gn.x, gn.y, gn.z};
        f3 pt{gp.x, gp.y, gp.z};
        float d = gp.w;
        f3 rA = sub3(pt, ldpos(S, a));
        f3 rB = bb >= 0 ? sub3(pt, ldpos(S, bb)) : f3{0.0f, 0.0f, 0.0f};
        f3 ex = fabsf(n.x) < 0.9f ? f3{1.0f, 0.0f, 0.0f} : f3{0.0f, 1.0f, 0.0f};
        f3 t = cross3(n, ex);
        float tl = sqrtf(dot3(t, t));
        f3 t1{t.x / tl, t.y / tl, t.z / tl};
        f3 t2 = cross3(n, t1);
        // effective masses along n, t1, t2, once per substep
        float kN = eff_mass(S, a, bb, rA, rB, n);
        float kT1 = eff_mass(S, a, bb, rA, rB, t1);
        float kT2 = eff_mass(S, a, bb, rA, rB, t2);
        float vn0 = dot3(n, rel_vel(S, a, bb, rA, rB));
        float vmin;
        if (d >= 0.0f) {
            vmin = -d / h;
        } else {
            float pen = -d - sc.slop;
            vmin = (sc.beta * (pen > 0.0f ? pen : 0.0f)) / h;
        }
        if (d < 0.0f && vn0 < -sc.rest_thr) {
            float vb = -sc.restitution * vn0;
            if (vb > vmin) vmin = vb;
        }
        r.g(F_N) = make_float4(n.x, n.y, n.z, kN);
        r.g(F_RA) = make_float4(rA.x, rA.y, rA.z, vmin);
        r.g(F_RB) = make_float4(rB.x, rB.y, rB.z, 0.0f);     // LN = 0
        r.g(F_T1) = make_float4(t1.x, t1.y, t1.z, kT1);
        r.g(F_T2) = make_float4(t2.x, t2.y, t2.z, kT2);
        r.g(F_P) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);      // LT1 = 0
        r.g(F_LA) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);     // LT2 = 0
    }
    __syncthreads();

    // 4. Jacobi iterations
    for (int it = 0; it < sc.iterations; it++) {
        for (int c = tid; c < nc; c += kT) {
            Rec r = C.rec(c);
            const float4 gn = r.g(F_N), ga = r.g(F_RA), gb = r.g(F_RB), g1 = r.g(F_T1), g2 = r.g(F_T2);
            const float l1 = r.g(F_P).w, l2 = r.g(F_LA).w;
            const int ab = __float_as_int(r.g(F_LB).w);
            const int a = ab & 0xffff, bb = (ab >> 16) - 1;
            f3 n{gn.x, gn.y, gn.z}, t1{g1.x, g1.y, g1.z}, t2{g2.x, g2.y, g2.z};
            f3 rA{ga.x, ga.y, ga.z}, rB{gb.x, gb.y, gb.z};
            f3 vr = rel_vel(S, a, bb, rA, rB);
            float vn = dot3(n, vr);
            float ln = gb.w;
            // the impulse updates divide by the effective mass as defined;
            // a precomputed reciprocal rounds differently, and in settled
            // piles one ulp there grows to ~1e-4 rad/s within a step
            float dl = (ga.w - vn) / gn.w;
            float lnew = ln + dl;
            if (!(lnew > 0.0f)) lnew = 0.0f;
            float dln = lnew - ln;
            r[F_LN] = lnew;
            float vt1 = dot3(t1, vr), vt2 = dot3(t2, vr);
            float a1 = l1 - vt1 / g1.w;
            float a2 = l2 - vt2 / g2.w;
            float lim = sc.mu * lnew;
            float m2 = a1 * a1 + a2 * a2;
            if (m2 > lim * lim) {
                float s = lim / sqrtf(m2);
                a1 = a1 * s;
                a2 = a2 * s;
            }
            float dl1 = a1 - l1, dl2 = a2 - l2;
            f3 P{(dln * n.x + dl1 * t1.x) + dl2 * t2.x, (dln * n.y + dl1 * t1.y) + dl2 * t2.y,
                 (dln * n.z + dl1 * t1.z) + dl2 * t2.z};
            const f3 LA = cross3(rA, P);
            r.g(F_P) = make_float4(P.x, P.y, P.z, a1);
            r.g(F_LA) = make_float4(LA.x, LA.y, LA.z, a2);
            if (bb >= 0) {
                const f3 LB = cross3(rB, P);
                r.g(F_LB) = make_float4(LB.x, LB.y, LB.z, __int_as_float(ab));
            }
        }
        __syncthreads();
        // per-body sums in ascending contact order, applied at once: unit u
        // is body (u / 64) * 32 + u % 32 and half (u / 32) % 2 -- the impulse
        // sum and linear velocity (0), or the moment sum and angular
        // velocity (1); consecutive lanes take consecutive bodies.  The B
        // side of a contact enters with the opposite sign.
        for (int u = tid; u < 2 * ((N + 31) & ~31); u += kT) {
            const int half = (u >> 5) & 1;
            const int i = ((u >> 6) << 5) + (u & 31);
            if (i >= N) continue;
            auto load = [&](int ent, float& x, float& y, float& z) {
                Rec r = C.rec(ent >> 1);
                const bool side = ent & 1;
                const float4 v = r.g(half == 0 ? F_P : (side ? F_LB : F_LA));
                x = v.x;
                y = v.y;
                z = v.z;
                if (side) {
                    x = -x;
                    y = -y;
                    z = -z;
                }
            };
            float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
            const int k1 = S.loff[i + 1];
            int k = S.loff[i];
            // loads of four entries are independent: issue them together,
            // then add in list order
            for (; k + 4 <= k1; k += 4) {
                float x[4], y[4], z[4];
#pragma unroll
                for (int q = 0; q < 4; q++) load(lists[k + q], x[q], y[q], z[q]);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    s0 = s0 + x[q];
                    s1 = s1 + y[q];
                    s2 = s2 + z[q];
                }
            }
            for (; k < k1; k++) {
                float x, y, z;
                load(lists[k], x, y, z);
                s0 = s0 + x;
                s1 = s1 + y;
                s2 = s2 + z;
            }
            if (half == 0) {
                const float im = S.IM(i);
                S.V(0, i) = S.V(0, i) + sc.omega * (im * s0);
                S.V(1, i) = S.V(1, i) + sc.omega * (im * s1);
                S.V(2, i) = S.V(2, i) + sc.omega * (im * s2);
            } else {
                const f3 dw = imul(S, i, f3{s0, s1, s2});
                S.W(0, i) = S.W(0, i) + sc.omega * dw.x;
                S.W(1, i) = S.W(1, i) + sc.omega * dw.y;
                S.W(2, i) = S.W(2, i) + sc.omega * dw.z;
            }
        }
        __syncthreads();
    }

}

// ---- hull contacts (sc.hulls) ------------------------------------------
// A hull body is the convex hull of its unit mesh scaled by its radius s
// (body-frame vertices s v_k, face planes n_f . x = s o_f from the mesh's
// planes); the pair tests treat a box as the polytope of its 8 corners and
// 6 faces.  Hull contacts follow all others: the plane contacts of the
// hulls (bodies in order, vertices in mesh order; none for a hull whose
// centre is at least its radius plus the margin above the plane), then the
// pairs (i, j), i < j, with a hull that pass the bounding-sphere test, in
// lexicographic order: a sphere's centre against the hull's deepest face,
// or the two polytopes (face separating-axis test, reference and incident
// face, Sutherland-Hodgman clipping).  Each such unit is worked by one warp.

// A box's face loops (corners in sign-bit order), counter-clockwise seen
// from outside: +x, -x, +y, -y, +z, -z.
__constant__ signed char kBoxLoop[24] = {1, 3, 7, 5, 0, 4, 6, 2, 2, 6, 7, 3, 0, 1, 5, 4, 4, 5, 7, 6, 0, 2, 3, 1};

struct Poly {
    bool hull;
    int nv, nf;
    const float4* v;      // hull: unit-mesh vertices [nv] (x, y, z, 0)
    const float4* pl;     // hull: unit-mesh face planes [nf]
    const int32_t* tri;   // hull: mesh-local vertex indices [nf][3]
    float s;              // hull: radius
    float h0, h1, h2;     // box: half extents
};

__device__ __forceinline__ Poly poly_of(const DevBatch& b, const Bodies& S, int b0, int i) {
    Poly P;
    P.hull = S.TYPE(i) == kShapeHull;
    if (P.hull) {
        const int m = __ldg(b.mesh_id + b0 + i);
        const int v0 = __ldg(b.mesh_vert_off + m), t0 = __ldg(b.mesh_tri_off + m);
        P.nv = __ldg(b.mesh_vert_off + m + 1) - v0;
        P.nf = __ldg(b.mesh_tri_off + m + 1) - t0;
        P.v = b.mesh_vert4 + v0;
        P.pl = b.mesh_plane + t0;
        P.tri = b.mesh_tris + 3 * (size_t)t0;
        P.s = S.D(0, i);
        P.h0 = P.h1 = P.h2 = 0.0f;
    } else {
        P.nv = 8;
        P.nf = 6;
        P.v = nullptr;
        P.pl = nullptr;
        P.tri = nullptr;
        P.s = 0.0f;
        P.h0 = S.D(0, i);
        P.h1 = S.D(1, i);
        P.h2 = S.D(2, i);
    }
    return P;
}

// body-frame vertex k
__device__ __forceinline__ f3 poly_x(const Poly& P, int k) {
    if (P.hull) {
        const float4 q = __ldg(P.v + k);
        return f3{P.s * q.x, P.s * q.y, P.s * q.z};
    }
    return f3{(k & 1) ? P.h0 : -P.h0, (k & 2) ? P.h1 : -P.h1, (k & 4) ? P.h2 : -P.h2};
}

// body-frame face plane f: outward unit normal, offset
__device__ __forceinline__ float4 poly_plane(const Poly& P, int f) {
    if (P.hull) {
        const float4 q = __ldg(P.pl + f);
        return make_float4(q.x, q.y, q.z, P.s * q.w);
    }
    const int ax = f >> 1;
    const float sg = (f & 1) ? -1.0f : 1.0f;
    return make_float4(ax == 0 ? sg : 0.0f, ax == 1 ? sg : 0.0f, ax == 2 ? sg : 0.0f,
                       ax == 0 ? P.h0 : (ax == 1 ? P.h1 : P.h2));
}

// vertex k of face f's loop, -1 past its end
__device__ __forceinline__ int poly_loop(const Poly& P, int f, int k) {
    if (P.hull) return k < 3 ? __ldg(P.tri + 3 * f + k) : -1;
    return kBoxLoop[4 * f + k];
}

__device__ __forceinline__ f3 poly_world(const Bodies& S, int i, const Poly& P, int k) {
    return add3(rmul(S, i, poly_x(P, k)), ldpos(S, i));
}

// Warp-wide maximum (minimum) of (value, index) pairs, the lowest index
// among equal values; lanes without a candidate hold index -1.
__device__ __forceinline__ void warp_best(float& v, int& k, bool want_max) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(kFull, v, o);
        const int ok = __shfl_xor_sync(kFull, k, o);
        const bool better = want_max ? ov > v : ov < v;
        if (ok >= 0 && (k < 0 || better || (ov == v && ok < k))) {
            v = ov;
            k = ok;
        }
    }
}

// Largest separation of polytope b from polytope a along a's face normals,
// sep_f = (min_v m . x_v + n . (p_b - p_a)) - offset_f with n = R_a n_f and
// m = R_b^T n, and its face (the first on ties).  Whole warp, a face per
// lane.  A box's minimum over its corners (+-h0, +-h1, +-h2) is taken in
// closed form: every product m_k (+-h_k) is +-(m_k h_k) exactly and
// rounding is monotonic, so the least of the eight sums ((p0 + p1) + p2) is
// the one with every term negative.
__device__ __forceinline__ float warp_face_separation(const Bodies& S, int a, const Poly& Pa, int b, const Poly& Pb,
                                                      int& face) {
    const int lane = threadIdx.x & 31;
    const f3 d = sub3(ldpos(S, b), ldpos(S, a));
    float best = 0.0f;
    int bf = -1;
    for (int f = lane; f < Pa.nf; f += 32) {
        const float4 pl = poly_plane(Pa, f);
        const f3 n = rmul(S, a, f3{pl.x, pl.y, pl.z});
        const f3 m = rtmul(S, b, n);
        float lo;
        if (!Pb.hull) {
            lo = (-fabsf(m.x * Pb.h0) - fabsf(m.y * Pb.h1)) - fabsf(m.z * Pb.h2);
        } else {
            // the minimum does not depend on the order of the vertices: four
            // vertices' loads are issued together
            lo = dot3(m, poly_x(Pb, 0));
            int v = 1;
#pragma unroll 1
            for (; v + 4 <= Pb.nv; v += 4) {
                f3 x[4];
#pragma unroll
                for (int u = 0; u < 4; u++) x[u] = poly_x(Pb, v + u);
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const float t = dot3(m, x[u]);
                    if (t < lo) lo = t;
                }
            }
#pragma unroll 1
            for (; v < Pb.nv; v++) {
                const float t = dot3(m, poly_x(Pb, v));
                if (t < lo) lo = t;
            }
        }
        const float sep = (lo + dot3(n, d)) - pl.w;
        if (bf < 0 || sep > best) {
            best = sep;
            bf = f;
        }
    }
    warp_best(best, bf, true);
    face = bf;
    return best;
}

// Contacts of polytope pair (i, j), i < j (see the oracle's reading):
// reference face of the larger separation (i's unless j's is larger by more
// than 1e-5 m), incident face of the other body (least n_g . n_ref, the
// first on ties), the incident loop clipped by the reference face's side
// planes, and each clipped point whose distance above the reference plane
// is below the margin, in order: normal n_ref from j to i, point the clipped
// point (at most 8 points are kept: rounding on nearly collinear points
// could add some to a convex polygon).  The warp works the face searches
// and the clipping, and with kWrite
// writes the contacts from index base.  Returns the contact count (every
// lane).
template <bool kWrite>
__device__ __forceinline__ int polytope_pair(const DevBatch& bt, const Bodies& S, const Contacts& C, int b0, int i, int j,
                                          float margin, int base, int cmax, bool& ovf, int* meta) {
    const int lane = threadIdx.x & 31;
    const Poly Pi = poly_of(bt, S, b0, i), Pj = poly_of(bt, S, b0, j);
    if (Pi.nv == 0 || Pi.nf == 0 || Pj.nv == 0 || Pj.nf == 0) return 0;   // an empty mesh has no contacts
    // the face searches of the counting pass are kept (meta: ref_j | fr << 1
    // | fq << 16, or -1 without contacts) and reused by the writing pass
    bool ref_j;
    int fr, fq;
    if (kWrite && meta) {
        const int mt = *meta;
        if (mt < 0) return 0;
        ref_j = mt & 1;
        fr = (mt >> 1) & 0x7fff;
        fq = mt >> 16;
    } else {
        int fi, fj;
        const float si = warp_face_separation(S, i, Pi, j, Pj, fi);
        // no contacts whatever j's separation when i's is at least the
        // margin: the reference separation is then si, or sj > si + 1e-5
        if (!(si < margin)) {
            if (meta && lane == 0) *meta = -1;
            return 0;
        }
        const float sj = warp_face_separation(S, j, Pj, i, Pi, fj);
        ref_j = sj > si + 1e-5f;
        if (!((ref_j ? sj : si) < margin)) {
            if (meta && lane == 0) *meta = -1;
            return 0;
        }
        fr = ref_j ? fj : fi;
        fq = -1;
    }
    const int r = ref_j ? j : i, q = ref_j ? i : j;
    const Poly& Pr = ref_j ? Pj : Pi;
    const Poly& Pq = ref_j ? Pi : Pj;
    const float4 plr = poly_plane(Pr, fr);
    const f3 nr = rmul(S, r, f3{plr.x, plr.y, plr.z});
    if (fq < 0) {
        float lo = 0.0f;
        for (int g = lane; g < Pq.nf; g += 32) {
            const float4 pg = poly_plane(Pq, g);
            const float t = dot3(rmul(S, q, f3{pg.x, pg.y, pg.z}), nr);
            if (fq < 0 || t < lo) {
                lo = t;
                fq = g;
            }
        }
        warp_best(lo, fq, false);
        if (meta && lane == 0) *meta = (ref_j ? 1 : 0) | (fr << 1) | (fq << 16);
    }
    // Sutherland-Hodgman across the lanes: lane k holds point k of the
    // polygon (k < np <= 8); per side plane each lane emits its point when
    // inside and the crossing point of its edge (k, k + 1) when the edge
    // crosses, at the positions of the sequential algorithm (ballot prefix
    // counts; positions past 8 dropped), and lane j gathers emission j
    const unsigned lt = (1u << lane) - 1u;
    f3 P{0.0f, 0.0f, 0.0f};
    int np = 0;
    while (np < 4 && poly_loop(Pq, fq, np) >= 0) np++;
    if (lane < np) P = poly_world(S, q, Pq, poly_loop(Pq, fq, lane));
    const int nloop = poly_loop(Pr, fr, 3) >= 0 ? 4 : 3;
    f3 RV{0.0f, 0.0f, 0.0f};   // lane e: vertex e of the reference loop
    if (lane < nloop) RV = poly_world(S, r, Pr, poly_loop(Pr, fr, lane));
    for (int e = 0; e < nloop && np > 0; e++) {
        const int e1 = (e + 1) % nloop;
        const f3 va{__shfl_sync(kFull, RV.x, e), __shfl_sync(kFull, RV.y, e), __shfl_sync(kFull, RV.z, e)};
        const f3 vb{__shfl_sync(kFull, RV.x, e1), __shfl_sync(kFull, RV.y, e1), __shfl_sync(kFull, RV.z, e1)};
        const f3 sn = cross3(sub3(vb, va), nr);
        const float so = dot3(sn, va);
        const int nxt = lane + 1 < np ? lane + 1 : 0;
        const f3 P1{__shfl_sync(kFull, P.x, nxt), __shfl_sync(kFull, P.y, nxt), __shfl_sync(kFull, P.z, nxt)};
        const bool live = lane < np;
        const float dp = dot3(sn, P) - so, dq = dot3(sn, P1) - so;
        const bool in0 = live && dp <= 0.0f;
        const bool cross = live && ((dp <= 0.0f) != (dq <= 0.0f));
        f3 I{0.0f, 0.0f, 0.0f};
        if (cross) {
            const float t = dp / (dp - dq);
            I = f3{P.x + t * (P1.x - P.x), P.y + t * (P1.y - P.y), P.z + t * (P1.z - P.z)};
        }
        const unsigned bin = __ballot_sync(kFull, in0), bcr = __ballot_sync(kFull, cross);
        const int pos = __popc(bin & lt) + __popc(bcr & lt);   // this lane's first emission
        const int nout = min(8, __popc(bin) + __popc(bcr));
        const bool emits = in0 || cross;
        // emission j comes from the last emitting lane whose first emission is <= j
        unsigned mine = 0u;
#pragma unroll
        for (int jj = 0; jj < 8; jj++) {
            const unsigned m = __ballot_sync(kFull, emits && pos <= jj);
            if (lane == jj) mine = m;
        }
        const int src = mine ? 31 - __clz(mine) : 0;
        const int spos = __shfl_sync(kFull, pos, src);
        const bool sin0 = __shfl_sync(kFull, in0 ? 1 : 0, src) != 0;
        const f3 SP{__shfl_sync(kFull, P.x, src), __shfl_sync(kFull, P.y, src), __shfl_sync(kFull, P.z, src)};
        const f3 SI{__shfl_sync(kFull, I.x, src), __shfl_sync(kFull, I.y, src), __shfl_sync(kFull, I.z, src)};
        const bool first = lane == spos && sin0;   // the source's own point, else its crossing point
        if (lane < nout) P = first ? SP : SI;
        np = nout;
    }
    const float off = dot3(nr, f3{__shfl_sync(kFull, RV.x, 0), __shfl_sync(kFull, RV.y, 0),
                                  __shfl_sync(kFull, RV.z, 0)});
    const f3 n = ref_j ? nr : f3{-nr.x, -nr.y, -nr.z};
    const float dd = dot3(nr, P) - off;
    const bool hit = lane < np && dd < margin;
    const unsigned bh = __ballot_sync(kFull, hit);
    if (kWrite && hit) {
        const int idx = base + __popc(bh & lt);
        if (idx < cmax) put_contact(C, idx, i, j, n, P, dd);
        else ovf = true;
    }
    return __popc(bh);
}

// One hull unit (code: i | j << 16, j = 0xffff for hull i on the plane) by
// a warp: its contact count, and with kWrite its contacts from index base.
template <bool kWrite>
__device__ __forceinline__ int hull_unit(const DevBatch& bt, const Bodies& S, const Contacts& C, int b0, int code,
                                      float margin, int base, int cmax, bool& ovf, int* meta) {
    const int lane = threadIdx.x & 31;
    const int i = code & 0xffff, j = (code >> 16) & 0xffff;
    if (j == 0xffff) {   // the hull's vertices below the margin
        const Poly P = poly_of(bt, S, b0, i);
        const f3 up{0.0f, 0.0f, 1.0f};
        int cnt = 0;
        for (int k0 = 0; k0 < P.nv; k0 += 32) {
            const int k = k0 + lane;
            f3 w{0.0f, 0.0f, 0.0f};
            bool hit = false;
            if (k < P.nv) {
                w = poly_world(S, i, P, k);
                hit = w.z < margin;
            }
            const unsigned m = __ballot_sync(kFull, hit);
            if (kWrite && hit) {
                const int idx = base + cnt + __popc(m & ((1u << lane) - 1u));
                if (idx < cmax) put_contact(C, idx, i, -1, up, w, w.z);
                else ovf = true;
            }
            cnt += __popc(m);
        }
        return cnt;
    }
    const bool sphere_j = S.TYPE(j) != kShapeHull && S.TYPE(j) != kShapeBox;
    const bool sphere_i = S.TYPE(i) != kShapeHull && S.TYPE(i) != kShapeBox;
    if (!sphere_i && !sphere_j) return polytope_pair<kWrite>(bt, S, C, b0, i, j, margin, base, cmax, ovf, meta);
    // a sphere's centre against the hull's deepest face
    const int sp = sphere_j ? j : i, hb = sphere_j ? i : j;
    const Poly P = poly_of(bt, S, b0, hb);
    if (P.nf == 0) return 0;   // an empty mesh has no contacts
    const f3 c = ldpos(S, sp);
    const f3 x = rtmul(S, hb, sub3(c, ldpos(S, hb)));
    float D = 0.0f;
    int f = -1;
    for (int g = lane; g < P.nf; g += 32) {
        const float4 pl = poly_plane(P, g);
        const float dd = dot3(f3{pl.x, pl.y, pl.z}, x) - pl.w;
        if (f < 0 || dd > D) {
            D = dd;
            f = g;
        }
    }
    warp_best(D, f, true);
    const float d = D - S.D(0, sp);
    if (!(d < margin)) return 0;
    if (kWrite && lane == 0) {
        const float4 pl = poly_plane(P, f);
        f3 nb = rmul(S, hb, f3{pl.x, pl.y, pl.z});
        const f3 pt{c.x - nb.x * D, c.y - nb.y * D, c.z - nb.z * D};
        if (sphere_j) nb = f3{-nb.x, -nb.y, -nb.z};   // from the sphere (j) to the hull (i)
        if (base < cmax) put_contact(C, base, i, j, nb, pt, d);
        else ovf = true;
    }
    return 1;
}

// The hull contacts of a substep (see above), appended at nc: rounds of
// kPairChunk candidate units (the N bodies, then the N (N - 1) / 2 pairs);
// the round's units are listed in order (plist), each warp counts the
// contacts of its units (pitem), a scan gives their first indices, and the
// warps write them.  Whole CTA; plist and pitem are free at this point.
__device__ __forceinline__ void hull_pass(const DevBatch& bt, const Bodies& S, const Contacts& C, int b0, int N,
                                       int* plist, unsigned short* pitem, int* meta, int nmeta, ScanBuf& wsum,
                                       float margin, bool plane, int cmax, int& nc, bool& ovf) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int total = N + N * (N - 1) / 2;
    constexpr int per = kPairChunk / kT;
    for (int k0 = 0; k0 < total; k0 += kPairChunk) {
        unsigned passmask = 0;
        int npass = 0;
        int codes[per];
#pragma unroll
        for (int r = 0; r < per; r++) {
            const int u = k0 + tid * per + r;
            codes[r] = 0;
            if (u >= total) continue;
            bool pass;
            if (u < N) {
                pass = plane && S.TYPE(u) == kShapeHull && S.P(2, u) - S.BR(u) < margin;
                codes[r] = u | (0xffff << 16);
            } else {
                int i, j;
                pair_of_index(u - N, N, i, j);
                pass = (S.TYPE(i) == kShapeHull || S.TYPE(j) == kShapeHull) && broad(S, i, j, margin);
                codes[r] = i | (j << 16);
            }
            if (pass) {
                passmask |= 1u << r;
                npass++;
            }
        }
        int nu;
        int o = block_excl_scan(npass, wsum, nu);
#pragma unroll
        for (int r = 0; r < per; r++)
            if (passmask & (1u << r)) plist[o++] = codes[r];
        __syncthreads();
        for (int q = warp; q < nu; q += kT / 32) {
            const int c = hull_unit<false>(bt, S, C, b0, plist[q], margin, 0, cmax, ovf, q < nmeta ? meta + q : nullptr);
            if (lane == 0) pitem[q] = (unsigned short)min(c, 0xffff);
        }
        __syncthreads();
        // first contact of each unit (counts and indices beyond the u16 range
        // are past any contact capacity: those contacts overflow)
        int sum = 0;
#pragma unroll
        for (int r = 0; r < per; r++) {
            const int q = tid * per + r;
            if (q < nu) sum += pitem[q];
        }
        int nct;
        int run = block_excl_scan(sum, wsum, nct);
#pragma unroll
        for (int r = 0; r < per; r++) {
            const int q = tid * per + r;
            if (q < nu) {
                const int c = pitem[q];
                pitem[q] = (unsigned short)min(run, 0xffff);
                run += c;
            }
        }
        __syncthreads();
        for (int q = warp; q < nu; q += kT / 32)
            hull_unit<true>(bt, S, C, b0, plist[q], margin, nc + pitem[q], cmax, ovf, q < nmeta ? meta + q : nullptr);
        nc += nct;
        __syncthreads();   // plist and pitem are rewritten by the next round
    }
}

// kFeat: the optional contact tests compiled in (kFeatEdges: box-box
// edge-edge contacts, kFeatHulls: hull contacts); sc.edges and sc.hulls
// decide at run time.  Without them the code is left out, and its register
// pressure.
template <int kFeat>
__device__ __forceinline__ void sim_env(const DevBatch& b, int e, int nsteps, const float* __restrict__ force, int slot0,
                                     int smem_per_env, int NB) {
    const SimConst& sc = b.sc;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    const int b0 = b.body_off[e];
    const int N = b.body_off[e + 1] - b0;
    const int B = b.B;
    // the range must lie in the batch and fit the shared-memory layout sized
    // for NB bodies (the library's own batches always do; a caller-supplied
    // one may not): otherwise skip the environment before touching anything
    if (b0 < 0 || N < 0 || N > NB || b0 > B - N) {
        if (tid == 0) atomicOr(b.flags + e, (unsigned)VUDA_FLAG_BAD_RANGE);
        return;
    }
    int cmax = sc.mcpb * N;
    const int cmax_nb = sc.mcpb * NB;

    Bodies S;
    float* fp = reinterpret_cast<float*>(smem);
    S.base = fp; fp += kBW * NB;
    int* ip = reinterpret_cast<int*>(fp);
    S.loff = ip; ip += NB + 1;
    int* qcnt = ip; ip += kParts * NB;   // [kParts][NB] contacts of each body in each part of the list
    int* plist = ip; ip += kPairChunk;   // units (passing pairs or plane bodies) of the current round
    unsigned short* pitem = reinterpret_cast<unsigned short*>(ip); ip += kPairChunk / 2;   // their first item
    ScanBuf wsum{ip, 0}; ip += 2 * (kT / 32);
    unsigned short* ptab = reinterpret_cast<unsigned short*>(ip); ip += 4 * NB;   // [8 NB] plane items
    unsigned short* lists = reinterpret_cast<unsigned short*>(ip);
    const size_t fixed = phys_fixed_bytes(NB, cmax_nb);
    // while contacts are generated the list area (2 cmax_nb u16) holds the
    // edge-test results of a round's first passing pairs, 32 bytes each
    float4* edge_slots = reinterpret_cast<float4*>((reinterpret_cast<uintptr_t>(lists) + 15) & ~(uintptr_t)15);
    const int nedge_slots = (int)((4 * (size_t)cmax_nb - 12) / 32);
    Contacts C;
    C.s = reinterpret_cast<float*>(smem + fixed);
    int capS = (int)((smem_per_env - (long)fixed) / (kCS * 4));
    if (capS > cmax) capS = cmax;
    if (capS < 0) capS = 0;
    C.cap = capS;
    C.g = b.spill + (size_t)b.spill_off[e] * kCS;
    // without a spill area the capacity is what shared memory holds
    // (contacts beyond it are dropped in order and flagged as overflow)
    if (b.spill == nullptr) cmax = capS;

    for (int i = tid; i < N; i += kT) {
        int g = b0 + i;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            S.P(k, i) = b.pos[k * B + g];
            S.V(k, i) = b.vel[k * B + g];
            S.W(k, i) = b.ang[k * B + g];
            S.D(k, i) = b.dims[k * B + g];
            S.II(k, i) = b.ii[k * B + g];
        }
#pragma unroll
        for (int k = 0; k < 4; k++) S.Q(k, i) = b.quat[k * B + g];
        S.IM(i) = b.im[g];
        int t = b.type[g];
        S.TYPE(i) = t;
        S.BR(i) = t == kShapeBox
                        ? sqrtf((S.D(0, i) * S.D(0, i) + S.D(1, i) * S.D(1, i)) + S.D(2, i) * S.D(2, i))
                        : S.D(0, i);
    }
    __syncthreads();
    // hull contacts only where the environment has a hull (shapes do not
    // change during the launch)
    bool hulls = (kFeat & kFeatHulls) && sc.hulls;
    if (kFeat & kFeatHulls) {
        bool mine = false;
        for (int i = tid; i < N; i += kT) mine = mine || S.TYPE(i) == kShapeHull;
        hulls = __syncthreads_or(hulls && mine) != 0;
    }
    // plane contact items in canonical order, fixed for the launch (shapes
    // do not change): one per sphere, the eight corners of a box in sign-bit
    // order, bodies in order
    int nplane = 0;
    for (int i0 = 0; i0 < N; i0 += kT) {
        const int i = i0 + tid;
        const int nsub = i < N ? (is_box(S, i) ? 8 : (hulls && S.TYPE(i) == kShapeHull ? 0 : 1)) : 0;
        int tot;
        const int ex = block_excl_scan(nsub, wsum, tot);
        for (int k = 0; k < nsub; k++) ptab[nplane + ex + k] = (unsigned short)((i << 3) | k);
        nplane += tot;
    }

    bool ovf = false;
    int nc = 0;
    const float h = sc.h;
    const bool edges = (kFeat & kFeatEdges) && sc.edges;
    const int kBoxItems = edges ? 17 : 16;   // narrow-phase items of a box-box pair
    const int npairs = N * (N - 1) / 2;
    const f3 up{0.0f, 0.0f, 1.0f};
    for (int step = 0; step < nsteps; step++) {
        for (int ss = 0; ss < sc.substeps; ss++) {
            // 1. velocities, rotation, world inverse inertia
            for (int i = tid; i < N; i += kT) {
                float im = S.IM(i);
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    float f = force ? force[k * B + b0 + i] : 0.0f;
                    S.V(k, i) = S.V(k, i) + h * (sc.g[k] + f * im);
                }
                float w = S.Q(0, i), x = S.Q(1, i), y = S.Q(2, i), z = S.Q(3, i);
                float R[9];
                R[0] = 1.0f - 2.0f * (y * y + z * z);
                R[1] = 2.0f * (x * y - w * z);
                R[2] = 2.0f * (x * z + w * y);
                R[3] = 2.0f * (x * y + w * z);
                R[4] = 1.0f - 2.0f * (x * x + z * z);
                R[5] = 2.0f * (y * z - w * x);
                R[6] = 2.0f * (x * z - w * y);
                R[7] = 2.0f * (y * z + w * x);
                R[8] = 1.0f - 2.0f * (x * x + y * y);
                float ib0 = S.II(0, i), ib1 = S.II(1, i), ib2 = S.II(2, i);
#pragma unroll
                for (int k = 0; k < 9; k++) S.Rm(k, i) = R[k];
                if (sc.gyro && S.TYPE(i) == kShapeBox) gyroscopic(S, i, R, ib0, ib1, ib2, h);
#pragma unroll
                for (int r = 0; r < 3; r++)
#pragma unroll
                    for (int c = 0; c < 3; c++)
                        S.I(3 * r + c, i) = ((R[3 * r] * ib0) * R[3 * c] + (R[3 * r + 1] * ib1) * R[3 * c + 1]) +
                                            (R[3 * r + 2] * ib2) * R[3 * c + 2];
            }
            // per-part contact counts of this substep's lists start at zero
            for (int i = tid; i < kParts * NB; i += kT) qcnt[i] = 0;
            __syncthreads();

            // 2a. plane contacts: the launch's plane items (one per sphere, a
            // box's corners in sign-bit order, bodies in order), hits
            // compacted in item order
            nc = 0;
            if (sc.plane) {
                // two items per thread (u0 + tid and u0 + kT + tid), compacted
                // in item order by one scan of both hit counts
                for (int u0 = 0; u0 < nplane; u0 += 2 * kT) {
                    bool hit[2];
                    int bi[2];
                    f3 pt[2];
                    float d[2];
#pragma unroll
                    for (int q = 0; q < 2; q++) {
                        const int u = u0 + q * kT + tid;
                        hit[q] = false;
                        bi[q] = 0;
                        pt[q] = f3{0.0f, 0.0f, 0.0f};
                        d[q] = 0.0f;
                        if (u < nplane) {
                            const int pe = ptab[u];
                            bi[q] = pe >> 3;
                            if (is_box(S, bi[q])) {
                                pt[q] = box_corner(S, bi[q], pe & 7);
                                d[q] = pt[q].z;
                            } else {
                                float r = S.D(0, bi[q]);
                                f3 p = ldpos(S, bi[q]);
                                d[q] = p.z - r;
                                pt[q] = f3{p.x, p.y, p.z - r};
                            }
                            hit[q] = d[q] < sc.margin;
                        }
                    }
                    int t2;
                    const int ex2 = block_excl_scan((hit[0] ? 1 : 0) | (hit[1] ? 0x10000 : 0), wsum, t2);
                    const int n0 = t2 & 0xffff;
#pragma unroll
                    for (int q = 0; q < 2; q++)
                        if (hit[q]) {
                            const int idx = nc + (q == 0 ? (ex2 & 0xffff) : n0 + (ex2 >> 16));
                            if (idx < cmax) put_contact(C, idx, bi[q], -1, up, pt[q], d[q]); else ovf = true;
                        }
                    nc += n0 + (t2 >> 16);
                }
            }
            // 2b. pairs in (i, j) order, kPairChunk candidates per round
            for (int k0 = 0; k0 < npairs; k0 += kPairChunk) {
                const int per = kPairChunk / kT;   // consecutive candidates per thread
                int kbeg = k0 + tid * per;
                int pi = 0, pj = 0;
                if (kbeg < npairs) pair_of_index(kbeg, N, pi, pj);
                unsigned passmask = 0;
                int npass = 0, nsub = 0;
                {
                    int i = pi, j = pj;
                    for (int r = 0; r < per; r++) {
                        if (kbeg + r < npairs) {
                            // pairs with a hull come after all others (hull_pass)
                            if (!(hulls && (S.TYPE(i) == kShapeHull || S.TYPE(j) == kShapeHull)) &&
                                broad(S, i, j, sc.margin)) {
                                passmask |= 1u << r;
                                npass++;
                                nsub += (is_box(S, i) && is_box(S, j)) ? kBoxItems : 1;
                            }
                            if (++j == N) { i++; j = i + 1; }
                        }
                    }
                }
                int tot;
                int ex = block_excl_scan(npass | (nsub << 16), wsum, tot);
                int np = tot & 0xffff, nitems = tot >> 16;
                {
                    int o = ex & 0xffff, it = ex >> 16;
                    int i = pi, j = pj;
                    for (int r = 0; r < per; r++) {
                        if (kbeg + r < npairs) {
                            if (passmask & (1u << r)) {
                                plist[o] = i | (j << 16);
                                pitem[o] = (unsigned short)it;
                                o++;
                                it += (is_box(S, i) && is_box(S, j)) ? kBoxItems : 1;
                            }
                            if (++j == N) { i++; j = i + 1; }
                        }
                    }
                }
                __syncthreads();
                if (edges) {
                    // the edge tests of the round's first box pairs, one thread
                    // each, into the per-body list scratch (unused until the
                    // solve); the item pass reads them (pairs beyond the slots,
                    // in crowded rounds only, are tested by their item)
                    edge_prepass<kFeat>(S, plist, 0, min(np, nedge_slots), edge_slots, sc.margin);
                    __syncthreads();
                }
                for (int u0 = 0; u0 < nitems; u0 += kT) {
                    int u = u0 + tid;
                    bool hit = false;
                    int i = 0, j = 0;
                    f3 n, pt;
                    float d = 0.0f;
                    if (u < nitems) {
                        int lo = 0, hi = np - 1;   // last passing pair whose first item is <= u
                        while (lo < hi) {
                            int mid = (lo + hi + 1) >> 1;
                            if (pitem[mid] <= u) lo = mid; else hi = mid - 1;
                        }
                        int pr = plist[lo];
                        i = pr & 0xffff;
                        j = pr >> 16;
                        const int sub = u - pitem[lo];
                        if ((kFeat & kFeatEdges) && sub == 16 && lo < nedge_slots) {   // a box pair's edge test, computed above
                            const float4 e0 = edge_slots[2 * lo], e1 = edge_slots[2 * lo + 1];
                            n = f3{e0.x, e0.y, e0.z};
                            d = e0.w;
                            pt = f3{e1.x, e1.y, e1.z};
                            hit = e1.w != 0.0f;
                        } else if ((kFeat & kFeatEdges) && sub == 16) {
                            hit = box_edge_edge<kFeat>(S, i, j, sc.margin, n, pt, d);
                        } else {
                            hit = pair_test(S, i, j, sub, sc.margin, n, pt, d);
                        }
                    }
                    int t2;
                    int ex2 = block_excl_scan(hit ? 1 : 0, wsum, t2);
                    if (hit) {
                        int idx = nc + ex2;
                        if (idx < cmax) put_contact(C, idx, i, j, n, pt, d); else ovf = true;
                    }
                    nc += t2;
                }
            }
            // the per-body list area (cmax_nb ints, unused until the solve)
            // keeps the hull units' face searches between the passes
            if (hulls)
                hull_pass(b, S, C, b0, N, plist, pitem, reinterpret_cast<int*>(lists), cmax_nb, wsum, sc.margin,
                          sc.plane != 0, cmax, nc, ovf);
            if (nc > cmax) nc = cmax;

            if (nc <= C.cap) solve_substep(SmemContacts{C.s}, S, qcnt, lists, wsum, nc, N, NB, sc, h);
            else solve_substep(C, S, qcnt, lists, wsum, nc, N, NB, sc, h);

            // 5. positions and orientations
            const float hh = 0.5f * h;
            for (int i = tid; i < N; i += kT) {
                S.P(0, i) = S.P(0, i) + h * S.V(0, i);
                S.P(1, i) = S.P(1, i) + h * S.V(1, i);
                S.P(2, i) = S.P(2, i) + h * S.V(2, i);
                float qw = S.Q(0, i), qx = S.Q(1, i), qy = S.Q(2, i), qz = S.Q(3, i);
                float wx = S.W(0, i), wy = S.W(1, i), wz = S.W(2, i);
                float dw = -((wx * qx + wy * qy) + wz * qz);
                float dx = qw * wx + (wy * qz - wz * qy);
                float dy = qw * wy + (wz * qx - wx * qz);
                float dz = qw * wz + (wx * qy - wy * qx);
                float nw = qw + hh * dw, nx = qx + hh * dx, ny = qy + hh * dy, nz = qz + hh * dz;
                float len = sqrtf(((nw * nw + nx * nx) + ny * ny) + nz * nz);
                S.Q(0, i) = nw / len; S.Q(1, i) = nx / len; S.Q(2, i) = ny / len; S.Q(3, i) = nz / len;
            }
            __syncthreads();
        }
        // pose of this step for the renderer
        float* pose = b.pose[(slot0 + step) & 1];
        for (int i = tid; i < N; i += kT) {
            int g = b0 + i;
            pose[0 * B + g] = S.P(0, i);
            pose[1 * B + g] = S.P(1, i);
            pose[2 * B + g] = S.P(2, i);
            pose[3 * B + g] = S.Q(0, i);
            pose[4 * B + g] = S.Q(1, i);
            pose[5 * B + g] = S.Q(2, i);
            pose[6 * B + g] = S.Q(3, i);
        }
    }
    for (int i = tid; i < N; i += kT) {
        int g = b0 + i;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            b.pos[k * B + g] = S.P(k, i);
            b.vel[k * B + g] = S.V(k, i);
            b.ang[k * B + g] = S.W(k, i);
        }
#pragma unroll
        for (int k = 0; k < 4; k++) b.quat[k * B + g] = S.Q(k, i);
    }
    int any_ovf = __syncthreads_or(ovf ? 1 : 0);
    if (tid == 0) {
        if (nsteps > 0) b.ncontacts[e] = nc;
        if (any_ovf) atomicOr(b.flags + e, (unsigned)VUDA_FLAG_CONTACT_OVERFLOW);
    }
}

// Copies a descriptor into shared memory with the whole CTA.
__device__ __forceinline__ void load_desc(DevBatch& dst, const DevBatch& src) {
    const int* a = reinterpret_cast<const int*>(&src);
    int* d = reinterpret_cast<int*>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(DevBatch) / 4); k += blockDim.x) d[k] = a[k];
}

// Single batch: CTA e steps environment e.
template <int kFeat>
__global__ void __launch_bounds__(kT, kMinCtas) sim_kernel(DevBatch b0, SimConst sc0, int nsteps,
                                                    const float* __restrict__ force, int slot0, int smem_per_env,
                                                    int NB) {
    __shared__ DevBatch sb;
    load_desc(sb, b0);
    __syncthreads();
    if (threadIdx.x == 0) sb.sc = sc0;
    __syncthreads();
    sim_env<kFeat>(sb, blockIdx.x, nsteps, force, slot0, smem_per_env, NB);
}

// Work list over several batches: persistent CTAs pull (batch, environment,
// pose slot) items from an atomic counter; one step each.
template <int kFeat>
__global__ void __launch_bounds__(kT, kMinCtas) sim_list_kernel(const DevBatch* __restrict__ descs,
                                                         const int2* __restrict__ items, int nitems, int* counter,
                                                         const float* __restrict__ force, int smem_per_env, int NB,
                                                         SmGate gate) {
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
        const int2 it = items[item];
        load_desc(sb, descs[it.x & kItemDescMask]);
        __syncthreads();
        sim_env<kFeat>(sb, it.y, 1, force, (it.x >> 24) & 1, smem_per_env, NB);
        __syncthreads();  // everyone is done with sb and s_item
    }
    if (threadIdx.x == 0) sm_gate_release(gate, s_gate);
}

}  // namespace

VUDA_SIM_NS_BEGIN

int phys_contacts_in_smem(int smem_per_env, int max_bodies, int mcpb) {
    size_t fixed = phys_fixed_bytes(max_bodies, mcpb * max_bodies);
    if ((size_t)smem_per_env < fixed) return 0;
    return (int)(((size_t)smem_per_env - fixed) / (kCS * 4));
}

int phys_min_smem_bytes(int max_bodies, int mcpb) { return (int)phys_fixed_bytes(max_bodies, mcpb * max_bodies); }

int phys_smem_bytes_default(int max_bodies, int mcpb) {
    size_t fixed = phys_fixed_bytes(max_bodies, mcpb * max_bodies);
    // room for 4.5 contacts per body in shared memory (a settled pile of
    // spheres and boxes has about 3.5), less the plane item table's 16 bytes
    // per body and 64 bytes; more spill to global memory.  With 32 bodies
    // this is 31,728 bytes (140 records), so that with the kernels' static
    // shared memory (the 480-byte batch descriptor) rounded up to the
    // allocation unit 7 environments fit on one SM: the descriptor must not
    // grow by more than 40 bytes
    size_t want = fixed + (size_t)kCS * 4 * ((9 * max_bodies + 1) / 2) - (size_t)16 * max_bodies - 64;
    if (want > 200 * 1024) want = 200 * 1024;
    if (want < fixed) want = fixed;
    return (int)align16(want);
}

int sim_ctas_per_sm(int smem_per_env) {
    int n = 0;
    // every variant has the same launch bounds (registers) and shared memory
    cudaFuncSetAttribute(sim_list_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_per_env);
    cudaFuncSetAttribute(sim_list_kernel<0>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sim_list_kernel<0>, kT, smem_per_env) != cudaSuccess)
        n = 1;
    return n > 0 ? n : 1;
}

int sim_smem_for_ctas(int ctas) {
    // the SM's shared memory shared by `ctas` CTAs, each also holding the
    // per-block reservation and the kernel's static shared memory (the batch
    // descriptor), with 256 bytes of slack each, rounded down to 1 KB (the
    // occupancy calculator's figure one allocation unit higher left one CTA
    // per SM in practice)
    int dev = 0, per_sm = 0, reserved = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) reserved = 1024;
    const int per_cta = per_sm / ctas - reserved - (int)sizeof(DevBatch) - 64 - 256;
    return per_cta > 0 ? per_cta & ~1023 : 0;
}

CtaFootprint sim_list_footprint(int smem_per_env) {
    cudaFuncAttributes fa[4]{};
    if (cudaFuncGetAttributes(&fa[0], sim_list_kernel<0>) != cudaSuccess ||
        cudaFuncGetAttributes(&fa[1], sim_list_kernel<1>) != cudaSuccess ||
        cudaFuncGetAttributes(&fa[2], sim_list_kernel<2>) != cudaSuccess ||
        cudaFuncGetAttributes(&fa[3], sim_list_kernel<3>) != cudaSuccess)
        return CtaFootprint{kT, 255, 227 * 1024};
    int regs = 0, smem = 0;
    for (const cudaFuncAttributes& a : fa) {
        regs = max(regs, a.numRegs);
        smem = max(smem, (int)a.sharedSizeBytes);
    }
    return CtaFootprint{kT, regs, smem + smem_per_env};
}

template <class K>
static cudaError_t prepare(K kernel, int smem_per_env) {
    // set on every launch: the attribute is tracked per context and the
    // kernel may be launched into different (green) contexts
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_per_env);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

template <int kFeat>
static cudaError_t launch_items_t(const DevBatch* descs, const int2* items, int nitems, int* counter, int grid,
                                  int smem_per_env, int max_bodies, const float* force, SmGate gate,
                                  cudaStream_t stream) {
    cudaError_t e = prepare(sim_list_kernel<kFeat>, smem_per_env);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
    if (e != cudaSuccess) return e;
    sim_list_kernel<kFeat><<<grid, kT, smem_per_env, stream>>>(descs, items, nitems, counter, force, smem_per_env,
                                                               max_bodies, gate);
    return cudaGetLastError();
}

cudaError_t launch_sim_items(const DevBatch* descs, const int2* items, int nitems, int* counter, int grid,
                             int smem_per_env, int max_bodies, const float* force, SmGate gate, int feat,
                             cudaStream_t stream) {
    if (nitems == 0) return cudaSuccess;
    switch (feat & (kFeatEdges | kFeatHulls)) {
        case 0: return launch_items_t<0>(descs, items, nitems, counter, grid, smem_per_env, max_bodies, force, gate, stream);
        case 1: return launch_items_t<1>(descs, items, nitems, counter, grid, smem_per_env, max_bodies, force, gate, stream);
        case 2: return launch_items_t<2>(descs, items, nitems, counter, grid, smem_per_env, max_bodies, force, gate, stream);
        default: return launch_items_t<3>(descs, items, nitems, counter, grid, smem_per_env, max_bodies, force, gate, stream);
    }
}

template <int kFeat>
static cudaError_t launch_env_t(const DevBatch& b, const SimConst& sc, int nsteps, const float* force, int slot0,
                                int smem_per_env, int max_bodies, cudaStream_t stream) {
    cudaError_t e = prepare(sim_kernel<kFeat>, smem_per_env);
    if (e != cudaSuccess) return e;
    sim_kernel<kFeat><<<b.E, kT, smem_per_env, stream>>>(b, sc, nsteps, force, slot0, smem_per_env, max_bodies);
    return cudaGetLastError();
}

cudaError_t launch_sim(const DevBatch& b, const SimConst& sc, int nsteps, const float* force, int slot0,
                       int smem_per_env, int max_bodies, cudaStream_t stream) {
    if (b.E == 0 || nsteps == 0) return cudaSuccess;
    size_t fixed = phys_fixed_bytes(max_bodies, sc.mcpb * max_bodies);
    if ((size_t)smem_per_env < fixed) smem_per_env = (int)fixed;
    switch (sim_features(sc)) {
        case 0: return launch_env_t<0>(b, sc, nsteps, force, slot0, smem_per_env, max_bodies, stream);
        case 1: return launch_env_t<1>(b, sc, nsteps, force, slot0, smem_per_env, max_bodies, stream);
        case 2: return launch_env_t<2>(b, sc, nsteps, force, slot0, smem_per_env, max_bodies, stream);
        default: return launch_env_t<3>(b, sc, nsteps, force, slot0, smem_per_env, max_bodies, stream);
    }
}

VUDA_SIM_NS_END

}  // namespace vuda
