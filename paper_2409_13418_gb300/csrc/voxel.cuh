// voxel.cuh -- dense voxel-grid occupancy: trilinear interpolation of a
// sample volume against iso, decided in float-float.
//
// Per axis u = (x - lo) / (hi - lo) * (dims - 1) (x - lo and hi - lo exact in
// float-float, the quotient to ~48 bits), clamped to [0, dims - 1]; cell
// i = min(floor(u), dims - 2), fraction u - i; lerps a + (b - a) f along x,
// then y, then z.  The decision phi > iso then equals the exact one except
// within ~1e-13 of iso.
#pragma once
#include "odc_device.cuh"

namespace odc {

__device__ __forceinline__ ff vox_lerp(ff a, ff b, ff f) { return ff_add(a, ff_mul(ff_sub(b, a), f)); }

struct VoxOcc {
    VoxDev d;
    __device__ __forceinline__ uint32_t operator()(float3 p) const {
        const float pc[3] = {p.x, p.y, p.z};
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
