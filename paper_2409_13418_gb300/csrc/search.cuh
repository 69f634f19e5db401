// search.cuh -- geometry of the 1D and 2D point searches (Sec. 5.1, 5.2,
// A.1.3, A.1.4), shared by the CSG kernels (whole search per thread) and the
// MLP wavefront kernels (one query batch per step).
//
// Face-local coordinates: a face normal to axis a spans u = axis (a+1)%3 and
// v = axis (a+2)%3 with the face as the unit square; world = X[i] + (X[i+1] -
// X[i]) * local per axis.  All positions are carried in float-float and
// rounded to float32 only to query phi.
#pragma once
#include "odc_device.cuh"

namespace odc {

struct ff2 {
    ff u, v;
};

__device__ __forceinline__ ff2 ff2_add(ff2 a, ff2 b) { return {ff_add(a.u, b.u), ff_add(a.v, b.v)}; }
__device__ __forceinline__ ff2 ff2_sub(ff2 a, ff2 b) { return {ff_sub(a.u, b.u), ff_sub(a.v, b.v)}; }
__device__ __forceinline__ ff2 ff2_scale(ff2 a, ff s) { return {ff_mul(a.u, s), ff_mul(a.v, s)}; }

// Line-binary search sample parameter s = R J / (N 2^b) (A.1.3).
__device__ __forceinline__ ff lbs_param(float R, uint32_t J, int n, int b) {
    ff num = two_prod(R, (float)J);
    float den = (float)(n << b);
    if ((n & (n - 1)) == 0) return ff_mulf(num, 1.0f / den);   // power of two: exact
    return ff_div(num, ff_make(den));
}

// One face segment of the 2D search.
struct FaceSeg {
    int a, b, c;          // face normal axis and in-face axes u = b, v = c
    int q[3];             // lowest vertex of the face
    float2 p1, p2;        // 1D points (face-local, exact dyadic)
    ff2 m;                // midpoint
    ff2 d;                // unit ray of step 1 (towards the label opposite to m's)
    ff2 u1;               // unit direction from p_e2 to p_e1 (ray r1 of step 2)
};

// Face-edge index -> face-local point at parameter tau along that edge.
__device__ __forceinline__ float2 face_edge_point(int fe, float tau) {
    switch (fe) {
        case 0: return make_float2(tau, 0.0f);
        case 1: return make_float2(1.0f, tau);
        case 2: return make_float2(tau, 1.0f);
        default: return make_float2(0.0f, tau);
    }
}

// Lowest vertex and axis of the global edge under face edge fe.
__device__ __forceinline__ void face_edge_global(const FaceSeg& F, int fe, int* x, int* y, int* z, int* axis) {
    int p[3] = {F.q[0], F.q[1], F.q[2]};
    if (fe == 1) p[F.b] += 1;
    if (fe == 2) p[F.c] += 1;
    *axis = (fe == 0 || fe == 2) ? F.b : F.c;
    *x = p[0];
    *y = p[1];
    *z = p[2];
}

// World point (float32) of face-local (u, v).
__device__ __forceinline__ float3 face_world(const GridDev& g, const FaceSeg& F, ff u, ff v) {
    float w[3];
    w[F.a] = g.X[F.a][F.q[F.a]];
    w[F.b] = axis_world_ff(g.X[F.b], F.q[F.b], u).hi;
    w[F.c] = axis_world_ff(g.X[F.c], F.q[F.c], v).hi;
    return make_float3(w[0], w[1], w[2]);
}

__device__ __forceinline__ float3 face_world2(const GridDev& g, const FaceSeg& F, ff2 p) {
    return face_world(g, F, p.u, p.v);
}

// Point p + s d.
__device__ __forceinline__ ff2 ray_point(ff2 p, ff2 d, ff s) { return ff2_add(p, ff2_scale(d, s)); }

// Set up a face segment: its two 1D points, midpoint and ray directions.
// ``lab4`` holds the face-corner labels, ``seg`` the two face edges.
__device__ __forceinline__ void face_setup(FaceSeg& F, int a, int x, int y, int z, int lab4, int fe1, int fe2,
                                           uint32_t T1, uint32_t T2, int k) {
    F.a = a;
    F.b = nxt3(a);
    F.c = prv3(a);
    F.q[0] = x;
    F.q[1] = y;
    F.q[2] = z;
    float inv = __int_as_float((127 - (k + 1)) << 23);   // 2^-(k+1)
    F.p1 = face_edge_point(fe1, (float)T1 * inv);
    F.p2 = face_edge_point(fe2, (float)T2 * inv);
    ff2 P1 = {ff_make(F.p1.x), ff_make(F.p1.y)}, P2 = {ff_make(F.p2.x), ff_make(F.p2.y)};
    F.m = {ff_mulf(ff_add(P1.u, P2.u), 0.5f), ff_mulf(ff_add(P1.v, P2.v), 0.5f)};
    ff2 dl = ff2_sub(P2, P1);
    ff2 d0 = {ff_neg(dl.v), dl.u};
    ff len = ff_sqrt(ff_add(ff_mul(d0.u, d0.u), ff_mul(d0.v, d0.v)));
    // in-side: the in-corner end of face edge fe1, as a unit step from its out-corner
    int cA = fe1, cB = (fe1 + 1) & 3;
    bool inA = (lab4 >> cA) & 1;
    // face corner positions (0,0),(1,0),(1,1),(0,1)
    const int cu[4] = {0, 1, 1, 0}, cv[4] = {0, 0, 1, 1};
    int wu = inA ? cu[cA] - cu[cB] : cu[cB] - cu[cA];
    int wv = inA ? cv[cA] - cv[cB] : cv[cB] - cv[cA];
    int sg = ff_sign(ff_add(ff_mulf(d0.u, (float)wu), ff_mulf(d0.v, (float)wv)));
    ff2 din = {ff_div(d0.u, len), ff_div(d0.v, len)};
    if (sg < 0) din = {ff_neg(din.u), ff_neg(din.v)};
    F.d = din;   // flipped later when m is inside
    ff2 e = ff2_sub(P1, P2);
    ff el = ff_sqrt(ff_add(ff_mul(e.u, e.u), ff_mul(e.v, e.v)));
    F.u1 = {ff_div(e.u, el), ff_div(e.v, el)};
}

// A 2D point as stored: float-float (u.hi, u.lo, v.hi, v.lo).
__device__ __forceinline__ float4 ff2_pack(ff2 p) { return make_float4(p.u.hi, p.u.lo, p.v.hi, p.v.lo); }

// Step 3 of the 2D search: intersection of lines (p_e1, q1) and (p_e2, q2);
// parallel lines give m.  Returns flags bit1 when parallel.
__device__ __forceinline__ float4 face_intersect(const FaceSeg& F, ff2 q1, ff2 q2, int* flags) {
    ff2 P1 = {ff_make(F.p1.x), ff_make(F.p1.y)}, P2 = {ff_make(F.p2.x), ff_make(F.p2.y)};
    ff2 r1 = ff2_sub(q1, P1), r2 = ff2_sub(q2, P2);
    ff det = ff_sub(ff_mul(r1.u, r2.v), ff_mul(r1.v, r2.u));
    float n1 = r1.u.hi * r1.u.hi + r1.v.hi * r1.v.hi;
    float n2 = r2.u.hi * r2.u.hi + r2.v.hi * r2.v.hi;
    float dh = fabsf(det.hi);
    if (dh * dh <= 1e-18f * n1 * n2) {
        *flags |= 2;
        return ff2_pack(F.m);
    }
    ff2 dp = ff2_sub(P2, P1);
    ff alpha = ff_div(ff_sub(ff_mul(dp.u, r2.v), ff_mul(dp.v, r2.u)), det);
    ff2 pf = ff2_add(P1, ff2_scale(r1, alpha));
    return ff2_pack(pf);
}

// Load face segment (fid, slot): its corner labels and pairing, the two 1D
// points from the 1D results T, and the search geometry.
__device__ __forceinline__ void load_face(const GridDev& g, const uint32_t* bits, const uint32_t* flips,
                                          const WordInfo* wi, const uint32_t* ebase, const uint32_t* T, int k,
                                          uint32_t fid, int slot, FaceSeg& F) {
    int x, y, z;
    vid_xyz(g, fid / 3u, &x, &y, &z);
    int a = (int)(fid % 3u);
    int b = nxt3(a), c = prv3(a);
    int lab4 = 0;
    for (int i = 0; i < 4; ++i) {
        int p[3] = {x, y, z};
        if (i == 1 || i == 2) p[b] += 1;
        if (i >= 2) p[c] += 1;
        lab4 |= (int)label_at(g, bits, p[0], p[1], p[2]) << i;
    }
    int seg[2][2];
    face_segments(lab4, flip_at(g, flips, a, x, y, z), seg);
    int fe1 = seg[slot][0], fe2 = seg[slot][1];
    F.a = a;
    F.b = b;
    F.c = c;
    F.q[0] = x;
    F.q[1] = y;
    F.q[2] = z;
    int ex, ey, ez, ea;
    face_edge_global(F, fe1, &ex, &ey, &ez, &ea);
    uint32_t T1 = T[edge_rank(g, wi, ebase, ex, ey, ez, ea)];
    face_edge_global(F, fe2, &ex, &ey, &ez, &ea);
    uint32_t T2 = T[edge_rank(g, wi, ebase, ex, ey, ez, ea)];
    face_setup(F, a, x, y, z, lab4, fe1, fe2, T1, T2, k);
}

}  // namespace odc
