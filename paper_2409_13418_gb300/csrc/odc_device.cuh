// odc_device.cuh -- device-side building blocks of the ODC path.
//
//  * float-float ("ff") arithmetic: a value hi + lo held in two floats with
//    about 48 significant bits (Dekker 1971; Knuth TAOCP vol. 2, 4.2.2).  The
//    search geometry of Sec. 5.1-5.2 runs in ff so that every query point,
//    once rounded to float32, is the point the double-precision definition
//    gives; FP64 is reserved for the QEF of Eq. 2.
//  * cube topology: corner/edge/face numbering, face pairing and the cycles
//    of a cell (A.1.1, Fig. A1), computed from the conventions, no tables.
//  * CSG occupancy: a float32 fast path with a rigorous error bound and an
//    ff re-decision for samples too close to a primitive's surface, so the
//    label equals the sign of the exact predicate at the float32 point.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "odc_internal.h"

namespace odc {

// ---------------------------------------------------------------- ff math
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_make(float a) { return {a, 0.0f}; }

__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, err};
}

__device__ __forceinline__ ff quick_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float err = __fsub_rn(b, __fsub_rn(s, a));
    return {s, err};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float err = __fmaf_rn(a, b, -p);
    return {p, err};
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = two_sum(x.hi, y.hi);
    ff t = two_sum(x.lo, y.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = quick_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }
__device__ __forceinline__ ff ff_abs(ff x) { return (x.hi < 0.0f || (x.hi == 0.0f && x.lo < 0.0f)) ? ff_neg(x) : x; }

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    ff p = two_prod(x.hi, y.hi);
    p.lo = __fmaf_rn(x.hi, y.lo, p.lo);
    p.lo = __fmaf_rn(x.lo, y.hi, p.lo);
    return quick_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ ff ff_mulf(ff x, float y) {
    ff p = two_prod(x.hi, y);
    p.lo = __fmaf_rn(x.lo, y, p.lo);
    return quick_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ ff ff_div(ff a, ff b) {
    float q1 = __fdiv_rn(a.hi, b.hi);
    ff r = ff_sub(a, ff_mulf(b, q1));
    float q2 = __fdiv_rn(r.hi, b.hi);
    r = ff_sub(r, ff_mulf(b, q2));
    float q3 = __fdiv_rn(r.hi, b.hi);
    ff q = quick_two_sum(q1, q2);
    return ff_add(q, ff_make(q3));
}

__device__ __forceinline__ ff ff_sqrt(ff a) {
    if (a.hi <= 0.0f) return {0.0f, 0.0f};
    float s = __fsqrt_rn(a.hi);
    ff r = ff_sub(a, two_prod(s, s));
    float corr = __fdiv_rn(r.hi, __fmul_rn(2.0f, s));
    return quick_two_sum(s, corr);
}

__device__ __forceinline__ int ff_sign(ff x) {
    if (x.hi > 0.0f) return 1;
    if (x.hi < 0.0f) return -1;
    return (x.lo > 0.0f) - (x.lo < 0.0f);
}

// --------------------------------------------------------------- topology
// corner index = dx + 2 dy + 4 dz; local edge 4a + o1 + 2 o2 (o1 along
// (a+1)%3, o2 along (a+2)%3); local face 2a + s spanning u = (a+1)%3,
// v = (a+2)%3, face corners (0,0),(1,0),(1,1),(0,1), face edge i joins
// face corners i and i+1.
__device__ __forceinline__ int nxt3(int a) { return a == 2 ? 0 : a + 1; }
__device__ __forceinline__ int prv3(int a) { return a == 0 ? 2 : a - 1; }

__device__ __forceinline__ int corner_of(int d0, int d1, int d2) { return d0 | (d1 << 1) | (d2 << 2); }

__device__ __forceinline__ int edge_corner0(int le) {
    int a = le >> 2, o1 = le & 1, o2 = (le >> 1) & 1;
    int d[3] = {0, 0, 0};
    d[nxt3(a)] = o1;
    d[prv3(a)] = o2;
    return corner_of(d[0], d[1], d[2]);
}

__device__ __forceinline__ int edge_corner1(int le) { return edge_corner0(le) | (1 << (le >> 2)); }

__device__ __forceinline__ int face_edge(int f, int i) {
    int a = f >> 1, s = f & 1, b = nxt3(a), c = prv3(a);
    switch (i) {
        case 0: return 4 * b + 0 + 2 * s;
        case 1: return 4 * c + s + 2;
        case 2: return 4 * b + 1 + 2 * s;
        default: return 4 * c + s;
    }
}

__device__ __forceinline__ int face_corner(int f, int i) {
    int a = f >> 1, s = f & 1, b = nxt3(a), c = prv3(a);
    int u = (i == 1 || i == 2), v = (i >= 2);
    int d[3];
    d[a] = s;
    d[b] = u;
    d[c] = v;
    return corner_of(d[0], d[1], d[2]);
}

// the two local faces holding local edge le
__device__ __forceinline__ int edge_face0(int le) { int a = le >> 2; return 2 * nxt3(a) + (le & 1); }
__device__ __forceinline__ int edge_face1(int le) { int a = le >> 2; return 2 * prv3(a) + ((le >> 1) & 1); }

// Face pairing (A.1.1 reading): returns the number of segments (0..2) and
// writes each as two face-edge indices, in slot order.  lab4 bit i = label of
// face corner i.  Ambiguous faces pair around the inside corners, or around
// the outside corners when flipped.
__device__ __forceinline__ int face_segments(int lab4, bool flip, int seg[2][2]) {
    int cross = 0, n = 0, idx[4];
    for (int i = 0; i < 4; ++i) {
        int li = (lab4 >> i) & 1, lj = (lab4 >> ((i + 1) & 3)) & 1;
        if (li != lj) { cross |= 1 << i; idx[n++] = i; }
    }
    if (n == 0) return 0;
    if (n == 2) {
        seg[0][0] = idx[0];
        seg[0][1] = idx[1];
        return 1;
    }
    // checkerboard: corners 0 and 2 share a label
    int want = flip ? 0 : 1;
    bool c0 = ((lab4 & 1) == want);   // corners 0, 2 are the paired ones
    if (c0) {   // segments around corners 0 (edges 3, 0) and 2 (edges 1, 2)
        seg[0][0] = 0; seg[0][1] = 3;
        seg[1][0] = 1; seg[1][1] = 2;
    } else {    // around corners 1 (edges 0, 1) and 3 (edges 2, 3)
        seg[0][0] = 0; seg[0][1] = 1;
        seg[1][0] = 2; seg[1][1] = 3;
    }
    return 2;
}

__device__ __forceinline__ int face_lab4(uint32_t cfg, int f) {
    int r = 0;
    for (int i = 0; i < 4; ++i) r |= ((cfg >> face_corner(f, i)) & 1) << i;
    return r;
}

__device__ __forceinline__ uint32_t nib(uint64_t w, int i) { return (uint32_t)(w >> (4 * i)) & 0xFu; }
__device__ __forceinline__ uint64_t set_nib(uint64_t w, int i, uint32_t v) {
    return (w & ~(0xFull << (4 * i))) | ((uint64_t)v << (4 * i));
}

// Cycles of a cell (A.1.1): 4-bit cycle index per local edge (0xF: not a
// crossing edge), numbered by increasing smallest local edge.
__device__ __forceinline__ uint64_t cell_cycles(uint32_t cfg, uint32_t flipmask, int* ncyc) {
    uint64_t p0 = ~0ull, p1 = ~0ull;
    for (int f = 0; f < 6; ++f) {
        int seg[2][2];
        int ns = face_segments(face_lab4(cfg, f), (flipmask >> f) & 1, seg);
        for (int s = 0; s < ns; ++s) {
            int e1 = face_edge(f, seg[s][0]), e2 = face_edge(f, seg[s][1]);
            if (nib(p0, e1) == 0xF) p0 = set_nib(p0, e1, e2); else p1 = set_nib(p1, e1, e2);
            if (nib(p0, e2) == 0xF) p0 = set_nib(p0, e2, e1); else p1 = set_nib(p1, e2, e1);
        }
    }
    uint64_t cyc = ~0ull;
    int n = 0;
    for (int le = 0; le < 12; ++le) {
        if (nib(p0, le) == 0xF || nib(cyc, le) != 0xF) continue;
        uint32_t prev = 0xF, cur = le;
        for (int guard = 0; guard < 13 && nib(cyc, cur) == 0xF; ++guard) {
            cyc = set_nib(cyc, cur, n);
            uint32_t a = nib(p0, cur), b = nib(p1, cur);
            uint32_t nx = (a != prev) ? a : b;
            prev = cur;
            cur = nx;
        }
        ++n;
    }
    *ncyc = n;
    return cyc;
}

// True when local face f has two segments on one cycle (manifold-fix test).
__device__ __forceinline__ bool face_same_cycle(uint32_t cfg, uint32_t flipmask, int f) {
    int seg[2][2];
    int ns = face_segments(face_lab4(cfg, f), (flipmask >> f) & 1, seg);
    if (ns != 2) return false;
    int n;
    uint64_t cyc = cell_cycles(cfg, flipmask, &n);
    return nib(cyc, face_edge(f, seg[0][0])) == nib(cyc, face_edge(f, seg[1][0]));
}

// Slot of the segment of local face f that holds local edge le.
__device__ __forceinline__ int face_slot_of(uint32_t cfg, uint32_t flipmask, int f, int le) {
    int seg[2][2];
    int ns = face_segments(face_lab4(cfg, f), (flipmask >> f) & 1, seg);
    for (int s = 0; s < ns; ++s)
        if (face_edge(f, seg[s][0]) == le || face_edge(f, seg[s][1]) == le) return s;
    return 0;
}

// Marching-cubes polygon order (Tab. A8's MC variants): the successor of
// crossing local edge le in its oriented cycle.  Each face boundary is walked
// counter-clockwise as seen from outside the cell (face-corner order for side
// 1, reversed for side 0); a segment runs from the face's out->in crossing to
// its in->out crossing, and le is the out->in crossing on exactly one of its
// two faces, where its successor is the other end of its segment.
__device__ __forceinline__ int mc_next(uint32_t cfg, uint32_t flipmask, int le) {
    for (int w = 0; w < 2; ++w) {
        const int f = w == 0 ? edge_face0(le) : edge_face1(le);
        const int lab4 = face_lab4(cfg, f);
        int seg[2][2];
        const int ns = face_segments(lab4, (flipmask >> f) & 1, seg);
        for (int s = 0; s < ns; ++s)
            for (int e = 0; e < 2; ++e) {
                const int x = seg[s][e];
                if (face_edge(f, x) != le) continue;
                const int a = (f & 1) ? x : ((x + 1) & 3), b = (f & 1) ? ((x + 1) & 3) : x;
                if (!((lab4 >> a) & 1) && ((lab4 >> b) & 1)) return face_edge(f, seg[s][1 - e]);
            }
    }
    return -1;
}

// ------------------------------------------------------------- grid access
__device__ __forceinline__ uint32_t label_at(const GridDev& g, const uint32_t* bits, int x, int y, int z) {
    return (bits[((size_t)z * g.nv[1] + y) * g.W + (x >> 5)] >> (x & 31)) & 1u;
}

__device__ __forceinline__ uint32_t cell_config(const GridDev& g, const uint32_t* bits, int x, int y, int z) {
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) c |= label_at(g, bits, x + (k & 1), y + ((k >> 1) & 1), z + ((k >> 2) & 1)) << k;
    return c;
}

__device__ __forceinline__ uint32_t flip_at(const GridDev& g, const uint32_t* flips, int a, int x, int y, int z) {
    return (flips[(((size_t)a * g.nv[2] + z) * g.nv[1] + y) * g.W + (x >> 5)] >> (x & 31)) & 1u;
}

__device__ __forceinline__ uint32_t cell_flipmask(const GridDev& g, const uint32_t* flips, int x, int y, int z) {
    uint32_t m = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        int a = f >> 1, s = f & 1;
        int q[3] = {x, y, z};
        q[a] += s;
        m |= flip_at(g, flips, a, q[0], q[1], q[2]) << f;
    }
    return m;
}

// rank lookups into the compacted lists (word = 32 vertices along x)
__device__ __forceinline__ size_t word_of(const GridDev& g, int x, int y, int z) {
    return ((size_t)z * g.nv[1] + y) * g.W + (x >> 5);
}

__device__ __forceinline__ uint32_t edge_rank(const GridDev& g, const WordInfo* wi, const uint32_t* ebase,
                                              int x, int y, int z, int a) {
    size_t w = word_of(g, x, y, z);
    const WordInfo& r = wi[w];
    uint32_t l = x & 31, below = (1u << l) - 1u;
    uint32_t n = ebase[w] + __popc(r.m[0] & below) + __popc(r.m[1] & below) + __popc(r.m[2] & below);
    if (a >= 1) n += (r.m[0] >> l) & 1u;
    if (a >= 2) n += (r.m[1] >> l) & 1u;
    return n;
}

__device__ __forceinline__ uint32_t face_rank(const GridDev& g, const WordInfo* wi, const uint32_t* fbase,
                                              int x, int y, int z, int a, int slot) {
    size_t w = word_of(g, x, y, z);
    const WordInfo& r = wi[w];
    uint32_t l = x & 31, below = (1u << l) - 1u;
    uint32_t n = fbase[w];
#pragma unroll
    for (int k = 0; k < 3; ++k) n += __popc(r.fhas[k] & below) + __popc(r.famb[k] & below);
    for (int k = 0; k < a; ++k) n += ((r.fhas[k] >> l) & 1u) + ((r.famb[k] >> l) & 1u);
    return n + slot;
}

__device__ __forceinline__ uint32_t cell_rank(const GridDev& g, const WordInfo* wi, const uint32_t* cbase,
                                              int x, int y, int z) {
    size_t w = word_of(g, x, y, z);
    uint32_t l = x & 31, below = (1u << l) - 1u;
    return cbase[w] + __popc(wi[w].cell & below);
}

__device__ __forceinline__ void vid_xyz(const GridDev& g, uint32_t v, int* x, int* y, int* z) {
    *x = (int)(v % (uint32_t)g.nv[0]);
    uint32_t t = v / (uint32_t)g.nv[0];
    *y = (int)(t % (uint32_t)g.nv[1]);
    *z = (int)(t / (uint32_t)g.nv[1]);
}

__device__ __forceinline__ void cid_xyz(const GridDev& g, uint32_t c, int* x, int* y, int* z) {
    *x = (int)(c % (uint32_t)g.n[0]);
    uint32_t t = c / (uint32_t)g.n[0];
    *y = (int)(t % (uint32_t)g.n[1]);
    *z = (int)(t / (uint32_t)g.n[1]);
}

// world coordinate X_a[i] + (X_a[i+1] - X_a[i]) u, in ff, rounded to float
__device__ __forceinline__ ff axis_world_ff(const float* X, int i, ff u) {
    ff span = two_sum(X[i + 1], -X[i]);
    return ff_add(ff_make(X[i]), ff_mul(span, u));
}

// --------------------------------------------------------------- CSG phi
// Sign of each primitive's predicate g at float32 point p: -1 inside, +1
// outside, 0 on the surface.  The float32 value decides when it clears a
// bound on its rounding error; otherwise the predicate is re-evaluated in
// ff from the exact differences p - c.
static constexpr float kU = 5.9604645e-8f;   // 2^-24

__device__ __forceinline__ ff ff_dot3f(ff dx, ff dy, ff dz, float a0, float a1, float a2) {
    return ff_add(ff_add(ff_mulf(dx, a0), ff_mulf(dy, a1)), ff_mulf(dz, a2));
}

static __device__ __noinline__ int prim_sign_ff(const PrimDev& P, float px, float py, float pz) {
    ff dx = two_sum(px, -P.c[0]), dy = two_sum(py, -P.c[1]), dz = two_sum(pz, -P.c[2]);
    ff d2 = ff_add(ff_add(ff_mul(dx, dx), ff_mul(dy, dy)), ff_mul(dz, dz));
    switch (P.type) {
        case PRIM_SPHERE: {
            return ff_sign(ff_sub(d2, two_prod(P.p[0], P.p[0])));
        }
        case PRIM_AABB:
        case PRIM_OBOX: {
            int any_pos = 0, all_neg = 1;
            for (int i = 0; i < 3; ++i) {
                ff l = (P.type == PRIM_AABB) ? (i == 0 ? dx : (i == 1 ? dy : dz))
                                             : ff_dot3f(dx, dy, dz, P.R[3 * i], P.R[3 * i + 1], P.R[3 * i + 2]);
                int s = ff_sign(ff_sub(ff_abs(l), ff_make(P.p[i])));
                any_pos |= (s > 0);
                all_neg &= (s < 0);
            }
            return any_pos ? 1 : (all_neg ? -1 : 0);
        }
        case PRIM_CYLINDER: {
            ff t = ff_dot3f(dx, dy, dz, P.R[6], P.R[7], P.R[8]);
            ff radial = ff_sub(ff_sub(d2, ff_mul(t, t)), two_prod(P.p[0], P.p[0]));
            ff axial = ff_sub(ff_abs(t), ff_make(P.p[1]));
            int sr = ff_sign(radial), sa = ff_sign(axial);
            if (sr > 0 || sa > 0) return 1;
            if (sr < 0 && sa < 0) return -1;
            return 0;
        }
        default: {   // torus
            ff t = ff_dot3f(dx, dy, dz, P.R[6], P.R[7], P.R[8]);
            ff R2 = two_prod(P.p[0], P.p[0]);
            ff q = ff_sub(ff_add(d2, R2), two_prod(P.p[1], P.p[1]));
            ff rho2 = ff_sub(d2, ff_mul(t, t));
            ff g = ff_sub(ff_mul(q, q), ff_mul(ff_mulf(R2, 4.0f), rho2));
            return ff_sign(g);
        }
    }
}

__device__ __forceinline__ int prim_sign(const PrimDev& P, float px, float py, float pz) {
    float dx = __fsub_rn(px, P.c[0]), dy = __fsub_rn(py, P.c[1]), dz = __fsub_rn(pz, P.c[2]);
    float d2 = dx * dx + dy * dy + dz * dz;
    switch (P.type) {
        case PRIM_SPHERE: {
            float r2 = P.p[0] * P.p[0];
            float g = d2 - r2;
            float b = 16.0f * kU * (d2 + r2) + 1e-30f;
            if (g > b) return 1;
            if (g < -b) return -1;
            break;
        }
        case PRIM_AABB:
        case PRIM_OBOX: {
            bool any_pos = false, all_neg = true;
            for (int i = 0; i < 3; ++i) {
                float l, mag;
                if (P.type == PRIM_AABB) {
                    l = (i == 0 ? dx : (i == 1 ? dy : dz));
                    mag = fabsf(l);
                } else {
                    float a0 = P.R[3 * i] * dx, a1 = P.R[3 * i + 1] * dy, a2 = P.R[3 * i + 2] * dz;
                    l = a0 + a1 + a2;
                    mag = fabsf(a0) + fabsf(a1) + fabsf(a2);
                }
                float t = fabsf(l) - P.p[i];
                float b = 8.0f * kU * (mag + P.p[i]) + 1e-30f;
                any_pos |= (t > b);
                all_neg &= (t < -b);
            }
            if (any_pos) return 1;
            if (all_neg) return -1;
            break;
        }
        case PRIM_CYLINDER: {
            float a0 = P.R[6] * dx, a1 = P.R[7] * dy, a2 = P.R[8] * dz;
            float t = a0 + a1 + a2;
            float bt = 8.0f * kU * (fabsf(a0) + fabsf(a1) + fabsf(a2)) + 1e-30f;
            float r2 = P.p[0] * P.p[0];
            float radial = d2 - t * t - r2;
            float br = 16.0f * kU * (d2 + t * t + r2) + 3.0f * fabsf(t) * bt + 1e-30f;
            float axial = fabsf(t) - P.p[1];
            float ba = bt + 4.0f * kU * P.p[1];
            if (radial > br || axial > ba) return 1;
            if (radial < -br && axial < -ba) return -1;
            break;
        }
        default: {
            float a0 = P.R[6] * dx, a1 = P.R[7] * dy, a2 = P.R[8] * dz;
            float t = a0 + a1 + a2;
            float bt = 8.0f * kU * (fabsf(a0) + fabsf(a1) + fabsf(a2)) + 1e-30f;
            float R2 = P.p[0] * P.p[0];
            float q = d2 + R2 - P.p[1] * P.p[1];
            float rho2 = d2 - t * t;
            float g = q * q - 4.0f * R2 * rho2;
            float b = 64.0f * kU * (q * q + 4.0f * R2 * (d2 + t * t) + fabsf(q) * (d2 + R2 + P.p[1] * P.p[1])) +
                      16.0f * R2 * fabsf(t) * bt + 1e-30f;
            if (g > b) return 1;
            if (g < -b) return -1;
            break;
        }
    }
    return prim_sign_ff(P, px, py, pz);
}

// Occupancy label of a CSG chain at float32 point p (Sec. 3 phi; union =
// or, difference = and strictly-outside).  ``cull`` holds per primitive the
// centre and a conservative squared bounding radius: outside it a primitive
// is strictly outside, which leaves the fold unchanged.
__device__ __forceinline__ uint32_t csg_label(const PrimDev* prims, const float4* cull, int n, float px,
                                              float py, float pz) {
    uint32_t in = 0;
    for (int i = 0; i < n; ++i) {
        float4 c = cull[i];
        float dx = px - c.x, dy = py - c.y, dz = pz - c.z;
        if (dx * dx + dy * dy + dz * dz > c.w) continue;
        int s = prim_sign(prims[i], px, py, pz);
        if (i == 0 || prims[i].op == OP_UNION) in |= (s < 0);
        else in &= (s > 0);
    }
    return in;
}

}  // namespace odc
