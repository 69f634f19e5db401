// csg_psi.cuh -- the implicit psi of a CSG source and its gradient, for
// the ablation's Manifold Dual Contouring variants (Sec. 4, Eqs. 1 and 3)
// and the CSG surface-distance measure.  psi is the min/max fold of the
// primitives' g (union: min(psi, g), difference: max(psi, -g)), every
// primitive evaluated (no culling), with the operation order written below;
// the units that include this header are compiled without FMA contraction,
// so F = float gives a defined FP32 value (the linear 1D point's integer
// depends on it) and F = double the FP64 one.  The gradient is the selected
// primitive's (strict comparisons: the earlier operand wins ties; the sign
// of 0 is +).
#pragma once
#include "odc_device.cuh"

namespace odc {

template <typename F>
__device__ __forceinline__ F psi_sgn(F v) { return v < F(0) ? F(-1) : F(1); }

// g of one primitive and, if grad is non-null, its gradient.
template <typename F>
__device__ F prim_g_t(const PrimDev& P, F x, F y, F z, F* grad) {
    const F dx = x - (F)P.c[0], dy = y - (F)P.c[1], dz = z - (F)P.c[2];
    const F p0 = (F)P.p[0], p1 = (F)P.p[1], p2 = (F)P.p[2];
    switch (P.type) {
        case PRIM_SPHERE: {
            if (grad) { grad[0] = F(2) * dx; grad[1] = F(2) * dy; grad[2] = F(2) * dz; }
            return ((dx * dx + dy * dy) + dz * dz) - p0 * p0;
        }
        case PRIM_AABB:
        case PRIM_OBOX: {
            F l[3];
            if (P.type == PRIM_AABB) {
                l[0] = dx; l[1] = dy; l[2] = dz;
            } else {
                for (int k = 0; k < 3; ++k)
                    l[k] = ((F)P.R[3 * k] * dx + (F)P.R[3 * k + 1] * dy) + (F)P.R[3 * k + 2] * dz;
            }
            const F v0 = fabs(l[0]) - p0, v1 = fabs(l[1]) - p1, v2 = fabs(l[2]) - p2;
            if (grad) {
                int k = 0;
                F best = v0;
                if (v1 > best) { k = 1; best = v1; }
                if (v2 > best) k = 2;
                const F s = psi_sgn(l[k]);
                for (int a = 0; a < 3; ++a)
                    grad[a] = P.type == PRIM_AABB ? (a == k ? s : F(0)) : s * (F)P.R[3 * k + a];
            }
            return fmax(fmax(v0, v1), v2);
        }
        case PRIM_CYLINDER:
        case PRIM_TORUS: {
            const F ax = (F)P.R[6], ay = (F)P.R[7], az = (F)P.R[8];
            const F tt = (ax * dx + ay * dy) + az * dz;
            const F d2 = (dx * dx + dy * dy) + dz * dz;
            const F rx = dx - tt * ax, ry = dy - tt * ay, rz = dz - tt * az;
            if (P.type == PRIM_CYLINDER) {
                const F g_r = ((d2 - tt * tt) - p0 * p0) / (F(2) * p0);
                const F axial = fabs(tt) - p1;
                if (grad) {
                    if (g_r >= axial) { grad[0] = rx / p0; grad[1] = ry / p0; grad[2] = rz / p0; }
                    else { const F s = psi_sgn(tt); grad[0] = s * ax; grad[1] = s * ay; grad[2] = s * az; }
                }
                return fmax(g_r, axial);
            }
            const F q = (d2 + p0 * p0) - p1 * p1;
            if (grad) {
                const F k8 = F(8) * p0 * p0;
                grad[0] = F(4) * q * dx - k8 * rx;
                grad[1] = F(4) * q * dy - k8 * ry;
                grad[2] = F(4) * q * dz - k8 * rz;
            }
            return q * q - ((F(4) * p0) * p0) * (d2 - tt * tt);
        }
    }
    if (grad) grad[0] = grad[1] = grad[2] = F(0);
    (void)p2;
    return F(0);
}

template <typename F>
__device__ F csg_psi(const PrimDev* prims, int n, F x, F y, F z, F* grad) {
    F gsel[3], gi[3];
    F psi = prim_g_t<F>(prims[0], x, y, z, grad ? gsel : nullptr);
    for (int i = 1; i < n; ++i) {
        const F g = prim_g_t<F>(prims[i], x, y, z, grad ? gi : nullptr);
        if (prims[i].op == OP_UNION) {
            if (g < psi) {
                psi = g;
                if (grad) for (int a = 0; a < 3; ++a) gsel[a] = gi[a];
            }
        } else if (-g > psi) {
            psi = -g;
            if (grad) for (int a = 0; a < 3; ++a) gsel[a] = -gi[a];
        }
    }
    if (grad) for (int a = 0; a < 3; ++a) grad[a] = gsel[a];
    return psi;
}

}  // namespace odc
