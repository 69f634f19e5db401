// voxel.cuh -- dense voxel-grid occupancy: trilinear interpolation of a
// sample volume against iso.
//
// Per axis u = (x - lo) / (hi - lo) * (dims - 1), clamped to [0, dims - 1];
// cell i = min(floor(u), dims - 2), fraction u - i; lerps a + (b - a) f along
// x, then y, then z.  A float32 evaluation decides first: its error is at
// most the fraction error (|du| <= 4 2^-24 (dims - 1), times the Lipschitz
// constant 2 vmax of each axis, vmax the largest corner magnitude) plus the
// rounding of seven lerps (< 30 2^-24 vmax); twice that bound, vmax (3e-6
// (dims - 1) + 4e-6), separates a sure decision from a near one.  Near ones
// are re-decided in float-float (x - lo and hi - lo exact, the quotient to
// ~48 bits), which equals the exact decision except within ~1e-13 of iso.
#pragma once
#include "odc_device.cuh"

namespace odc {

__device__ __forceinline__ ff vox_lerp(ff a, ff b, ff f) { return ff_add(a, ff_mul(ff_sub(b, a), f)); }

// Float32 sample coordinate along axis a: cell index c and fraction f of
// world coordinate x (the fast path's own rounding; the float-float path
// below decides whatever this path leaves undecided).
__device__ __forceinline__ void vox_axis32(const VoxDev& d, int a, float x, int* c, float* f) {
    const float top = (float)(d.dims[a] - 1);
    float u = (x - d.lo[a]) / d.rng_hi[a] * top;
    u = fminf(fmaxf(u, 0.0f), top);
    *c = min((int)u, d.dims[a] - 2);
    *f = u - (float)*c;
}

// The float32 trilinear value at cell (i) fractions (f), decided against iso
// when it lies beyond its rounding bound: 1 inside, 0 outside, -1 undecided.
__device__ __forceinline__ int vox_fast32(const VoxDev& d, const int (&i)[3], const float (&f)[3]) {
    const int dmax = max(max(2, d.dims[0]), max(d.dims[1], d.dims[2]));
    const size_t sy = (size_t)d.dims[0], sz = (size_t)d.dims[0] * d.dims[1];
    const float* b = d.v + (size_t)i[2] * sz + (size_t)i[1] * sy + (size_t)i[0];
    const float v0 = __ldg(b), v1 = __ldg(b + 1), v2 = __ldg(b + sy), v3 = __ldg(b + sy + 1);
    const float v4 = __ldg(b + sz), v5 = __ldg(b + sz + 1), v6 = __ldg(b + sz + sy), v7 = __ldg(b + sz + sy + 1);
    const float c00 = fmaf(v1 - v0, f[0], v0), c10 = fmaf(v3 - v2, f[0], v2);
    const float c01 = fmaf(v5 - v4, f[0], v4), c11 = fmaf(v7 - v6, f[0], v6);
    const float c0 = fmaf(c10 - c00, f[1], c00), c1 = fmaf(c11 - c01, f[1], c01);
    const float phi = fmaf(c1 - c0, f[2], c0);
    const float vmax = fmaxf(fmaxf(fmaxf(fabsf(v0), fabsf(v1)), fmaxf(fabsf(v2), fabsf(v3))),
                             fmaxf(fmaxf(fabsf(v4), fabsf(v5)), fmaxf(fabsf(v6), fabsf(v7))));
    const float bound = vmax * (3e-6f * (float)(dmax - 1) + 4e-6f);
    if (phi - d.iso > bound) return 1;
    if (d.iso - phi > bound) return 0;
    return -1;
}

struct VoxOcc {
    VoxDev d;
    __device__ __forceinline__ uint32_t operator()(float3 p) const {
        const float pc[3] = {p.x, p.y, p.z};
        {   // float32 fast path
            int i[3];
            float f[3];
            for (int a = 0; a < 3; ++a) vox_axis32(d, a, pc[a], &i[a], &f[a]);
            const int r = vox_fast32(d, i, f);
            if (r >= 0) return (uint32_t)r;
        }
        int i[3];
        ff f[3];
        for (int a = 0; a < 3; ++a) {
            const float top = (float)(d.dims[a] - 1);
            ff u = ff_div(ff_sub(ff_make(pc[a]), ff_make(d.lo[a])), ff{d.rng_hi[a], d.rng_lo[a]});
            u = ff_mulf(u, top);
            if (u.hi < 0.0f || (u.hi == 0.0f && u.lo < 0.0f)) u = ff_make(0.0f);
            if (u.hi > top || (u.hi == top && u.lo > 0.0f)) u = ff_make(top);
            int c = (int)floorf(u.hi);
            if ((float)c == u.hi && u.lo < 0.0f) --c;
            c = min(max(c, 0), d.dims[a] - 2);
            i[a] = c;
            f[a] = ff_sub(u, ff_make((float)c));
        }
        const size_t sx = 1, sy = (size_t)d.dims[0], sz = (size_t)d.dims[0] * d.dims[1];
        const float* b = d.v + (size_t)i[2] * sz + (size_t)i[1] * sy + (size_t)i[0];
        const ff c00 = vox_lerp(ff_make(__ldg(b)), ff_make(__ldg(b + sx)), f[0]);
        const ff c10 = vox_lerp(ff_make(__ldg(b + sy)), ff_make(__ldg(b + sy + sx)), f[0]);
        const ff c01 = vox_lerp(ff_make(__ldg(b + sz)), ff_make(__ldg(b + sz + sx)), f[0]);
        const ff c11 = vox_lerp(ff_make(__ldg(b + sz + sy)), ff_make(__ldg(b + sz + sy + sx)), f[0]);
        const ff phi = vox_lerp(vox_lerp(c00, c10, f[1]), vox_lerp(c01, c11, f[1]), f[2]);
        return ff_sign(ff_sub(phi, ff_make(d.iso))) > 0 ? 1u : 0u;
    }
};

}  // namespace odc
