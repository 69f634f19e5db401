// odc_internal.h -- structures shared by the host orchestrator and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

namespace odc {

// Message returned by odc_last_error() for the calling thread.
void set_last_error(const std::string& msg);

enum { PRIM_SPHERE = 0, PRIM_AABB = 1, PRIM_OBOX = 2, PRIM_CYLINDER = 3, PRIM_TORUS = 4 };
enum { OP_UNION = 0, OP_DIFFERENCE = 1 };

constexpr int kMaxRes = 1024;
constexpr int kMaxPrims = 4096;

// Grid geometry in device-friendly form.
struct GridDev {
    int n[3];          // cells per axis
    int nv[3];         // vertices per axis
    int W;             // 32-bit words per label row: ceil(nv[0] / 32)
    const float* X[3]; // per-axis float32 vertex coordinates (device)
};

// Per 32-vertex word of a label row: crossing masks of the vertex-owned
// edges (3 axes), faces with crossings and ambiguous faces (3 axes), and
// crossing cells whose lowest corner is the vertex.
struct WordInfo {
    uint32_t m[3];
    uint32_t fhas[3];
    uint32_t famb[3];
    uint32_t cell;
};

struct PrimDev {
    int type;
    int op;
    float c[3];
    float R[9];
    float p[4];
    float pad[2];
};
static_assert(sizeof(PrimDev) == 80, "PrimDev must match odc_csg_prim");

// Dense voxel volume on the device (trilinear occupancy against iso).
struct VoxDev {
    const float* v;       // values [nz][ny][nx]
    int dims[3];
    float lo[3];
    float rng_hi[3], rng_lo[3];   // hi - lo per axis as float-float (exact)
    float iso;
};

// Search parameters (device copy of odc_params).
// Kernel launches issued by the library (all streams, all contexts).
void note_launch();
long long launch_count();

// Decisions of one 2D search (exported for parity checks): the near-end
// parameters J of the three line-binary searches, the label of m, and
// whether each linear phase met a label change (bit0 step 1, bit1 ray r1,
// bit2 ray r2).
struct FaceDecisions {
    uint32_t Jq, J1, J2;
    uint8_t lab_m, found, pad0, pad1;
};

struct SearchParams {
    int steps_1d;
    int lin1, bin1;
    float range1;
    int lin2, bin2;
    float range2;
    int ic_split;
};

}  // namespace odc
