// qef.cu -- normals from 2D points (Sec. 5.3) and one QEF 3D point per
// cycle (Eq. 2), one thread per crossing cell.
//
// For every crossing edge e of a cycle, the two faces of the cell that hold
// e each carry the 2D point of the segment through e (stored float-float);
// the plane through p_e and those two points has normal n = (p_f1 - p_e) x
// (p_f2 - p_e) in cell-local units.  Each normal is a row of the QEF normal
// matrix and is formed in FP64 with it: QEF sum_e (n_e . (p - p_e))^2 is
// accumulated as A = sum n n^T, b = sum n (n . p_e) and solved about the mass point
// c of the cycle's 1D points: p = c + A^+ (b - A c), with A^+ the
// pseudo-inverse keeping eigenvalues >= 0.01 of the largest (cyclic Jacobi
// eigen-decomposition, FP64, in registers).  For the ablation's MDC variants
// the normal is grad psi at the 1D point instead (Eq. 3).
#include "kernels.h"
#include "odc_device.cuh"

namespace odc {

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (Golub & Van
// Loan, Sec. 8.5): A = V diag(w) V^T.
__device__ __forceinline__ void jacobi3(double a[3][3], double V[3][3], double w[3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 16; ++sweep) {
        double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (off <= 1e-34 * dia || off == 0.0) break;
        for (int p = 0; p < 2; ++p) {
            for (int q = p + 1; q < 3; ++q) {
                double apq = a[p][q];
                if (apq == 0.0) continue;
                double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                // A <- J^T A J on the symmetric matrix (Golub & Van Loan, Alg. 8.5.2):
                // t solves t^2 + 2 theta t - 1 = 0, so the (p, q) entry becomes 0
                const int r = 3 - p - q;
                a[p][p] -= t * apq;
                a[q][q] += t * apq;
                a[p][q] = a[q][p] = 0.0;
                const double arp = a[r][p], arq = a[r][q];
                a[r][p] = a[p][r] = c * arp - s * arq;
                a[r][q] = a[q][r] = s * arp + c * arq;
                for (int k = 0; k < 3; ++k) {   // V <- V J
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
        }
    }
    for (int i = 0; i < 3; ++i) w[i] = a[i][i];
}

__global__ void k_qef(GridDev g, const uint32_t* __restrict__ flips, const WordInfo* __restrict__ wi,
                      const uint32_t* __restrict__ ebase, const uint32_t* __restrict__ fbase,
                      const uint32_t* __restrict__ T, const float4* __restrict__ pf, const float3* __restrict__ gnorm,
                      const uint32_t* __restrict__ cells,
                      const uint8_t* __restrict__ configs, const unsigned long long* __restrict__ cycles,
                      const uint32_t* __restrict__ vbase, uint32_t nc, int k, float3* __restrict__ vlocal,
                      float3* __restrict__ vworld) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    int cp[3];
    cid_xyz(g, cells[i], &cp[0], &cp[1], &cp[2]);
    uint32_t cfg = configs[i];
    uint32_t fm = cell_flipmask(g, flips, cp[0], cp[1], cp[2]);
    uint64_t cyc = cycles[i];
    float inv = __int_as_float((127 - (k + 1)) << 23);
    int ncyc = 0;
    for (int le = 0; le < 12; ++le) ncyc = max(ncyc, nib(cyc, le) == 0xF ? 0 : (int)nib(cyc, le) + 1);
    for (int cy = 0; cy < ncyc; ++cy) {
        double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        double bv[3] = {0, 0, 0}, cs[3] = {0, 0, 0};
        int cnt = 0;
        for (int le = 0; le < 12; ++le) {
            if (nib(cyc, le) != (uint32_t)cy) continue;
            int a = le >> 2;
            int d0 = edge_corner0(le);
            int o[3] = {d0 & 1, (d0 >> 1) & 1, (d0 >> 2) & 1};
            const uint32_t er = edge_rank(g, wi, ebase, cp[0] + o[0], cp[1] + o[1], cp[2] + o[2], a);
            uint32_t te = T[er];
            double pe[3] = {(double)o[0], (double)o[1], (double)o[2]};
            pe[a] = (double)te * (double)inv;
            double pfs[2][3] = {{0, 0, 0}, {0, 0, 0}};
            for (int s = 0; s < 2 && !gnorm; ++s) {
                int f = s == 0 ? edge_face0(le) : edge_face1(le);
                int fa = f >> 1, fs = f & 1;
                int q[3] = {cp[0], cp[1], cp[2]};
                q[fa] += fs;
                int slot = face_slot_of(cfg, fm, f, le);
                float4 uv = pf[face_rank(g, wi, fbase, q[0], q[1], q[2], fa, slot)];
                pfs[s][fa] = (double)fs;
                pfs[s][nxt3(fa)] = (double)uv.x + (double)uv.y;
                pfs[s][prv3(fa)] = (double)uv.z + (double)uv.w;
            }
            // the plane's normal is a row of the QEF normal matrix: formed in FP64
            double v1[3] = {pfs[0][0] - pe[0], pfs[0][1] - pe[1], pfs[0][2] - pe[2]};
            double v2[3] = {pfs[1][0] - pe[0], pfs[1][1] - pe[1], pfs[1][2] - pe[2]};
            double n[3] = {v1[1] * v2[2] - v1[2] * v2[1], v1[2] * v2[0] - v1[0] * v2[2], v1[0] * v2[1] - v1[1] * v2[0]};
            if (gnorm) {   // Eq. 3: grad psi, as a normal in cell-local units
                const float3 gw = gnorm[er];
                const double gv[3] = {(double)gw.x, (double)gw.y, (double)gw.z};
                for (int j = 0; j < 3; ++j) n[j] = gv[j] * ((double)g.X[j][cp[j] + 1] - (double)g.X[j][cp[j]]);
            }
            for (int j = 0; j < 3; ++j) cs[j] += pe[j];
            ++cnt;
            double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            if (nn < 1e-12) continue;   // degenerate plane: dropped
            double nh[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
            double dp = nh[0] * pe[0] + nh[1] * pe[1] + nh[2] * pe[2];
            for (int r = 0; r < 3; ++r) {
                bv[r] += nh[r] * dp;
                for (int c = 0; c < 3; ++c) A[r][c] += nh[r] * nh[c];
            }
        }
        double cbar[3] = {cs[0] / cnt, cs[1] / cnt, cs[2] / cnt};
        double rhs[3];
        for (int r = 0; r < 3; ++r) rhs[r] = bv[r] - (A[r][0] * cbar[0] + A[r][1] * cbar[1] + A[r][2] * cbar[2]);
        double V[3][3], w[3];
        jacobi3(A, V, w);
        double wmax = fmax(fmax(w[0], w[1]), w[2]);
        double x[3] = {cbar[0], cbar[1], cbar[2]};
        if (wmax > 0.0) {
            double t[3];
            for (int j = 0; j < 3; ++j) {
                double proj = V[0][j] * rhs[0] + V[1][j] * rhs[1] + V[2][j] * rhs[2];
                t[j] = (w[j] >= 0.01 * wmax) ? proj / w[j] : 0.0;
            }
            for (int r = 0; r < 3; ++r) x[r] += V[r][0] * t[0] + V[r][1] * t[1] + V[r][2] * t[2];
        }
        uint32_t vid = vbase[i] + cy;
        vlocal[vid] = make_float3((float)x[0], (float)x[1], (float)x[2]);
        float wv[3];
        for (int r = 0; r < 3; ++r) {
            double x0 = g.X[r][cp[r]], x1 = g.X[r][cp[r] + 1];
            wv[r] = (float)(x0 + (x1 - x0) * x[r]);
        }
        vworld[vid] = make_float3(wv[0], wv[1], wv[2]);
    }
}

void launch_qef(const GridDev& g, const uint32_t* flips, const WordInfo* wi, const uint32_t* ebase,
                const uint32_t* fbase, const uint32_t* T, const float4* pf, const float3* gnorm, const uint32_t* cells,
                const uint8_t* configs, const unsigned long long* cycles, const uint32_t* vbase, uint32_t nc, int k,
                float3* vlocal, float3* vworld, cudaStream_t st) {
    if (nc) { k_qef<<<(nc + 127) / 128, 128, 0, st>>>(g, flips, wi, ebase, fbase, T, pf, gnorm, cells, configs, cycles,
                                                   vbase, nc, k, vlocal, vworld); note_launch(); }
}

}  // namespace odc
