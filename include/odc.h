/*
 * odc.h -- C ABI of the GB300 occupancy-based dual contouring (ODC) library.
 *
 * The library turns an occupancy function phi: R^3 -> {0 (out), 1 (in)} on a
 * uniform grid over a box into a triangle mesh, following "Occupancy-Based
 * Dual Contouring" (Hwang & Sung, SIGGRAPH Asia 2024): given phi and a grid
 * over the space P, extract a mesh of the boundary surface (Sec. 3).  Every
 * stage runs as a CUDA kernel for sm_103a on one GPU:
 *   grid occupancy (Sec. 3) -> compaction of crossing edges, faces and cells
 *   -> cycles per cell with the manifold fix (A.1.1) -> 1D binary search
 *   (Sec. 5.1) -> 2D line-binary search (Sec. 5.2, A.1.3, A.1.4) -> normals
 *   from 2D points (Sec. 5.3) -> one QEF 3D point per cycle (Eq. 2) -> quads
 *   split by convex/concave analysis (Sec. 5.4, A.1.5).
 *
 * Conventions
 *   - Grid: res[a] cells per axis; vertex coordinates x_i = fl32(lo + (hi -
 *     lo) i / res) per axis, computed in double and rounded to float.
 *   - phi is evaluated at the query point rounded to float32.  A point is
 *     inside only if occ > iso strictly (ties are outside).
 *   - Vertex id v = i + (res0+1) (j + (res1+1) k); edge and face ids are
 *     3 v + a for the edge along axis a from vertex v and the face normal to
 *     axis a whose lowest corner is v.
 *   - Output vertices are float32 [n_verts][3] world coordinates; triangles
 *     are int32 [n_tris][3], counter-clockwise seen from outside (A.1.5).
 *     Vertices are the 3D points in cell order (cycles by increasing smallest
 *     local edge), then the case-3 1D points in edge order; triangles are in
 *     edge order.  The same input gives byte-identical output.
 *
 * Ownership
 *   - A context owns one device, a stream (unless the caller passes one) and
 *     a device memory arena that grows on demand up to ``mem_budget`` bytes.
 *   - Source descriptors (primitives, weights) are HOST pointers; they are
 *     copied to the device inside odc_extract.
 *   - The mesh returned by odc_extract points into context memory; it stays
 *     valid until the next odc_extract on the same context, odc_mesh_release
 *     or odc_ctx_destroy.  odc_mesh_copy copies it into caller buffers.
 *
 * Errors
 *   - Every call returns an odc_status; no exception or exit crosses the
 *     ABI.  CUDA errors map to ODC_ERR_CUDA; odc_last_error() returns a
 *     thread-local message for the last failing call on this thread.
 *   - Invalid arguments (null pointers, res < 1 or res > 1024, lo >= hi,
 *     steps_1d outside [1, 20], unknown primitive types, n_prims outside
 *     [1, 4096], unsupported MLP shapes) return ODC_ERR_INVALID_ARG.
 *   - Exceeding mem_budget returns ODC_ERR_OOM.
 *   - Device-side waits are bounded; an expired wait returns ODC_ERR_TIMEOUT.
 */
#ifndef ODC_H
#define ODC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ODC_OK = 0,
    ODC_ERR_INVALID_ARG = 1,
    ODC_ERR_OOM = 2,
    ODC_ERR_CUDA = 3,
    ODC_ERR_TIMEOUT = 4,
    ODC_ERR_UNSUPPORTED = 5,
    ODC_ERR_INTERNAL = 6
} odc_status;

typedef struct odc_ctx odc_ctx;

/* Occupancy source kinds.  ODC_SRC_RESIDENT reuses the source last uploaded
 * to the context (by odc_source_upload or a previous odc_extract). */
enum { ODC_SRC_CSG = 0, ODC_SRC_MLP = 1, ODC_SRC_RESIDENT = 2, ODC_SRC_VOXEL = 3 };

/* CSG primitive types and operations (Sec. 3: any phi; CSG is a synthetic
 * stand-in for the paper's neural occupancies). */
enum { ODC_PRIM_SPHERE = 0, ODC_PRIM_AABB = 1, ODC_PRIM_OBOX = 2,
       ODC_PRIM_CYLINDER = 3, ODC_PRIM_TORUS = 4 };
enum { ODC_OP_UNION = 0, ODC_OP_DIFFERENCE = 1 };

/* One CSG primitive, 80 bytes.  d = x - center.
 *   sphere:   params = [r]                 inside iff |d|^2 < r^2
 *   aabb:     params = [ex, ey, ez]        inside iff |d_i| < e_i for all i
 *   obox:     params = [ex, ey, ez]        l_i = rot[i] . d, inside iff |l_i| < e_i
 *   cylinder: params = [r, hh], axis rot[2]  t = axis . d,
 *             inside iff |d|^2 - t^2 < r^2 and |t| < hh
 *   torus:    params = [R, r], axis rot[2]
 *             inside iff (|d|^2 + R^2 - r^2)^2 < 4 R^2 (|d|^2 - t^2)
 * The primitives are folded left to right: in = in || in_p (union) or
 * in = in && out_p (difference, out_p strictly outside); prims[0].op is
 * treated as a union. */
typedef struct {
    int32_t type;
    int32_t op;
    float center[3];
    float rot[9];      /* row-major 3x3, rows are the local axes */
    float params[4];
    float pad[2];
} odc_csg_prim;

/* MLP precisions.  ODC_PREC_FP8 runs an FP8 tensor-core pass (E4M3
 * activations and weights, per-layer power-of-two scales, FP32 accumulation,
 * tcgen05 kind::f8f6f4) ahead of the BF16 path: its logits within 2.5 of the
 * threshold (2.1 times its largest measured logit error against the FP32
 * network, 1.19 on 600 k points; median 0.14)
 * go on to the BF16 pass and then the same tiers, so every decision still
 * equals the FP32 plain path's.  ODC_PREC_SPLIT, ODC_PREC_F16 and
 * ODC_PREC_FP8_RAW (odc_eval_points only) evaluate every point with the
 * split-FP16 tensor-core network, the single-product FP16 network or the
 * FP8 pass, without band handling. */
enum { ODC_PREC_FP32 = 0, ODC_PREC_BF16 = 1, ODC_PREC_SPLIT = 2, ODC_PREC_F16 = 3, ODC_PREC_FP8 = 4,
       ODC_PREC_FP8_RAW = 5 };

/* Envelope MLP occupancy: occ(x) = sigmoid(env_scale (env_radius - |x| +
 * env_amp f(x))), f(x) = W_L relu(... relu(W_0 [latent, g(x)] + b_0) ...) + b_L,
 * g(x) = [sin(2 pi B x), cos(2 pi B x)].  All pointers are host float32
 * row-major: B [n_freq][3], W_0 [hidden][latent_dim + 2 n_freq],
 * W_1..W_{n_hidden-1} [hidden][hidden], W_{n_hidden} [1][hidden], biases
 * b_l [rows of W_l].  Supported: n_freq = 64, hidden = 256, n_hidden = 4,
 * latent_dim in {0, 128}.  With ODC_PREC_BF16 every decision whose BF16
 * occupancy lies within ``band`` of iso is re-evaluated so that its sign
 * equals the FP32 plain path's: first by a single-product FP16 tensor-core
 * pass (FP16 activations and weights w 2^s, FP32 accumulation), whose logits
 * within 0.025 of the threshold (2.7 times its measured logit error of
 * 0.0091) go on to a split-precision tensor-core pass
 * (operands split into FP16 hi + lo, three products per layer, FP32
 * accumulation of hi hi and of the lo corrections in separate accumulators),
 * then, for the logits still within ``split_zmargin`` of the threshold (0:
 * calibrated for each uploaded network, 2.5 times the largest split-tier
 * logit difference against the FP32 network on 65536 calibration points and
 * at least 1.2e-5; over eight networks of this shape that is about twice
 * the largest difference seen on 3 M points), by the FP32 network;
 * ``no_split`` nonzero sends every
 * band decision to the FP32 network directly.  A band of 0.03 (|z| < 0.12)
 * covers the measured BF16 logit error (0.063) twice over. */
typedef struct {
    int32_t n_freq;
    int32_t hidden;
    int32_t n_hidden;
    int32_t latent_dim;
    const float* B;
    const float* W[8];
    const float* b[8];
    const float* latent;
    float env_scale;
    float env_radius;
    float env_amp;
    int32_t precision;
    float band;
    int32_t no_split;
    float split_zmargin;
    int32_t flags;               /* ODC_MLP_REUPLOAD: prepare and upload the weights even when the
                                    context already holds the same ones (by default a context that
                                    holds the same B, W and b only refreshes the latent's folded bias);
                                    ODC_MLP_NO_F16_TIER: band decisions skip the FP16 tier and go
                                    to the split tier directly (same decisions, other cost);
                                    ODC_MLP_FP32_TILE(v): run the FP32 network with tile shape v
                                    (0..3) instead of the autotuner's pick -- every shape gives the
                                    same bits */
    float h16_zmargin;           /* logits of the FP16 tier within this of the threshold go on to the
                                    split tier (0: the default 0.025) */
    float split_acc_comp;        /* split tier: the layer sums of its tensor-core products are taken as
                                    (1 + c K / 256) times what the tensor core returns, undoing on
                                    average its accumulation, which rounds every MMA's sum toward
                                    zero.  0 (the default): c is calibrated for each uploaded network
                                    (its logit error against the FP32 network is fitted against the
                                    network output at two values of c on 65536 points, half of them
                                    on the surface shell 0.3 <= |x| <= 0.7, and c is set where the
                                    fit's slope vanishes; a few ms per upload of new weights); > 0:
                                    this c; < 0: none.  Must be below 1e-3. */
} odc_mlp;

/* The FP32 network has four tile shapes (warps x K chunk x chunks in flight:
 * 16x32x2, 16x16x3, 12x32x3, 8x32x3); the first upload on a device times
 * each on a calibration list and keeps the fastest (odc_stats.fp32_tile). */
enum { ODC_MLP_REUPLOAD = 1, ODC_MLP_NO_F16_TIER = 2 };
#define ODC_MLP_FP32_TILE(v) (((v) + 1) << 8)

/* Dense voxel-grid occupancy: values[k][j][i] (host float32, i fastest) are
 * samples at lo + (hi - lo) (i, j, k) / (dims - 1); phi(x) is their trilinear
 * interpolation with x clamped to the box, inside iff phi > iso.  The
 * decision is taken in float-float (~48 bits), so it equals the exact one
 * except within ~1e-13 of iso.  dims in [2, 2048] per axis, at most 2^31
 * samples, lo < hi. */
typedef struct {
    int32_t dims[3];
    float lo[3];
    float hi[3];
    const float* values;
} odc_voxels;

typedef struct {
    int32_t kind;                /* ODC_SRC_CSG, ODC_SRC_MLP, ODC_SRC_VOXEL or ODC_SRC_RESIDENT */
    int32_t n_prims;
    const odc_csg_prim* prims;   /* host, n_prims records (CSG) */
    const odc_mlp* mlp;          /* host (MLP) */
    const odc_voxels* voxels;    /* host (VOXEL) */
} odc_source;

typedef struct {
    float lo[3];
    float hi[3];
    int32_t res[3];
} odc_grid;

/* Search parameters; the paper's values are iso 0.5, k = 15 at 128^3
 * (Sec. 5.1), step 1 of the 2D search 4 samples + 11 bisections over
 * 0.8 cell, step 2 3 samples + 12 bisections over sqrt(2)/2 cell (A.1.4). */
typedef struct {
    float iso;
    int32_t steps_1d;
    int32_t s2d_lin1, s2d_bin1;
    float s2d_range1;
    int32_t s2d_lin2, s2d_bin2;
    float s2d_range2;
    int32_t ic_split;            /* 1: IC quad splitting (A.1.5); 0: first diagonal */
    int32_t flags;               /* ablation variants (ODC_ABL_*), 0 for ODC */
} odc_params;

/* Ablation variants (Sec. 6.3, Tab. 3), CSG sources only (they need the
 * implicit psi, the min/max fold of the primitives' g, and its gradient; an
 * MLP source returns ODC_ERR_UNSUPPORTED).  ODC_ABL_LINEAR_1D: 1D points by
 * Eq. 1 (psi interpolated linearly along the edge in FP32, rounded to the
 * 2^-(k+1)-edge lattice) instead of the binary search.
 * ODC_ABL_GRADIENT_NORMALS: grad psi at the 1D point as the QEF plane normal
 * (Eq. 3) instead of the 2D points; the 2D search is skipped.  With ic_split
 * = 0 both give Manifold Dual Contouring, ODC_ABL_GRADIENT_NORMALS alone its
 * "+1D search" row. */
enum { ODC_ABL_LINEAR_1D = 1, ODC_ABL_GRADIENT_NORMALS = 2 };

/* Marching-cubes polygonization through the 1D points (Tab. A8's "MC" rows),
 * any source: the mesh vertices are the 1D points of the crossing edges in
 * edge order, and every cycle of every crossing cell (the same A.1.1 cycles
 * and manifold fix) is a polygon fanned from its smallest local edge, cells
 * in cell order, counter-clockwise seen from outside; no 2D search, QEF or
 * quads.  With ODC_ABL_LINEAR_1D (CSG) it is plain marching cubes. */
enum { ODC_POLY_MC = 4 };

typedef struct {
    int64_t n_edges;             /* |E^S| crossing edges */
    int64_t n_face_segs;         /* 2D points (one per face segment) */
    int64_t n_cells;             /* |C^S| crossing cells */
    int64_t n_verts3;            /* 3D points (cycles) */
    int64_t n_case3;             /* quads split into 4 triangles */
    int64_t n_flips;             /* faces flipped by the manifold fix */
    int64_t fix_rounds;
    int64_t n_queries;           /* occupancy evaluations on the main path */
    int64_t n_requeries;         /* FP32 (SIMT) re-evaluations of band decisions */
    float stage_ms[8];           /* grid, compact, topology, 1D, 2D, QEF, quads, total */
    double mlp_flops;            /* algorithmic FLOPs of the FP32 (SIMT) network launches */
    float mlp_ms;                /* CUDA-event time of the FP32 network launches */
    int32_t n_launches;          /* kernel launches issued by this extract */
    int64_t mlp_launches;        /* FP32 network launches */
    double tc_flops;             /* algorithmic FLOPs of the BF16 tensor-core network launches */
    float tc_ms;                 /* CUDA-event time of the tensor-core network launches */
    int32_t pad_;
    int64_t tc_launches;         /* tensor-core network launches */
    double split_flops;          /* tensor-pipe FLOPs of the split-FP16 re-evaluation (3 products) */
    float split_ms;              /* CUDA-event time of the split-FP16 launches */
    int32_t pad2_;
    int64_t split_launches;
    int64_t n_split;             /* band decisions re-evaluated by the split-FP16 tier */
    int64_t fp32_tile;           /* FP32 network tile shape used (MLP sources; -1 otherwise) */
    double h16_flops;            /* algorithmic FLOPs of the FP16-tier launches */
    float h16_ms;                /* CUDA-event time of the FP16-tier launches */
    int32_t pad3_;
    int64_t h16_launches;
    int64_t n_h16;               /* band decisions re-evaluated by the FP16 tier */
    double fp8_flops;            /* algorithmic FLOPs of the FP8-pass launches (ODC_PREC_FP8) */
    float fp8_ms;                /* CUDA-event time of the FP8-pass launches */
    int32_t pad4_;
    int64_t fp8_launches;
    float split_zmargin;         /* the split tier's logit margin in this extract (MLP sources) */
    float split_acc_comp;        /* its accumulation compensation c (MLP sources) */
} odc_stats;

typedef struct {
    int64_t n_verts;
    int64_t n_tris;
    const float* d_verts;        /* device, context-owned */
    const int32_t* d_tris;       /* device, context-owned */
    odc_stats stats;
} odc_mesh;

/* Create a context on CUDA device ``device``; the arena may grow to
 * ``mem_budget`` bytes (0 = no limit).  *out is NULL on failure. */
odc_status odc_ctx_create(int device, size_t mem_budget, odc_ctx** out);

/* Device bytes the context holds now (arenas, merged slab mesh, network
 * weights and scratch), for memory accounting. */
odc_status odc_ctx_memory(odc_ctx* ctx, size_t* bytes);

/* Failure detection of the device pipelines (the paper has no counterpart:
 * its evaluations have no device-side waits).  ``ns`` limits, in
 * nanoseconds of device global time, every pipeline wait (an mbarrier
 * phase: a weight slice landing, an accumulator or activation tile ready)
 * of this context's single-CTA tensor-core kernels, the BF16 pass and the
 * FP16 tier of the BF16 path; 0 restores the default of 2 s.  ``d_gate``
 * (device int32, caller-owned, or NULL for none) holds those kernels
 * before their first tensor-core operation until *d_gate != 0, waiting
 * under the same limit: a go signal from other device work.  A wait that
 * runs out sets the kernel's abort flag: every role of the CTA stops
 * issuing, the weight loads and tensor-core operations already started are
 * waited for (shared memory and TMEM are released idle), and the call that
 * launched the kernel returns ODC_ERR_TIMEOUT with its outputs undefined;
 * the context stays usable.  A gate that nothing sets is how a test makes
 * a wait run out without a hung device. */
odc_status odc_ctx_set_wait_limit(odc_ctx* ctx, uint64_t ns, const int32_t* d_gate);

/* Destroy a context and free its device memory.  NULL is accepted. */
odc_status odc_ctx_destroy(odc_ctx* ctx);

/* Run the whole ODC path for one shape.  ``cuda_stream`` is a cudaStream_t
 * (NULL: the context's own stream).  Returns after the mesh is complete in
 * device memory (the counts are read back once).  Sec. 3 problem statement;
 * stages as listed at the top of this header. */
odc_status odc_extract(odc_ctx* ctx, const odc_source* src, const odc_grid* grid,
                       const odc_params* params, void* cuda_stream, odc_mesh* out);

/* ---- z-slab extraction (a grid cut into slabs of cell layers along z)
 *
 * A slab owns the cells of layers [z0, z1), their 3D points, the crossing
 * edges whose lower end lies in those layers and the quads (with IC case-3
 * edge points) of those edges (Sec. 4 "Polygonization", A.1.5).  It is
 * extracted on its layers plus ``halo`` layers each side (clamped to the
 * grid), with the whole grid's vertex coordinates, so that every value it
 * owns equals the whole-grid extraction's; halo >= 2 covers the manifold
 * fix and the face searches of its boundary cells.  The whole grid's mesh
 * numbers 3D points in cell order, then edge points in edge order, and
 * triangles in edge order, so a slab's owned part is three contiguous
 * ranges and the merged mesh equals the whole-grid mesh byte for byte.  The
 * manifold fix (A.1.1) is the one non-local step: its flips chain from cell
 * to cell, round by round, across any slab plane.  So the slabs take the
 * whole grid's flips, computed once from the whole grid's label words:
 * odc_grid_labels fills the label words of a range of vertex layers (each
 * slab, or each rank, its own), odc_manifold_flips runs the fix over the
 * complete words.  Label words: W = (res[0] + 32) / 32 words per row,
 * word (w, y, z) at (z (res[1] + 1) + y) W + w, bit x % 32 of word x / 32
 * set where the vertex is inside; flip words: three such planes sets
 * (one per face axis), 3 W (res[1] + 1) (res[2] + 1) words. */
typedef struct {
    int32_t z0, z1;              /* owned cell layers [z0, z1), 0 <= z0 < z1 <= res[2] */
    int32_t halo;                /* extra cell layers each side, >= 1 */
    const uint32_t* flips;       /* device: the whole grid's flip words (odc_manifold_flips), or NULL: the
                                    slab runs the manifold fix on its own window (see fix_near_plane) */
} odc_slab;

typedef struct {
    int64_t verts3_local;        /* 3D points of the slab extraction (its edge points follow them) */
    int64_t verts3_before;       /* its 3D points below layer z0 */
    int64_t verts3_owned;        /* 3D points of the owned cells */
    int64_t case3_before;        /* edge points of halo edges before the owned edges */
    int64_t case3_owned;         /* edge points of the owned edges */
    int64_t tris_before;         /* triangles of halo edges before the owned edges */
    int64_t tris_owned;          /* triangles of the owned edges */
    int64_t fix_near_plane;      /* without whole-grid flips: manifold-fix marks within two layers of an
                                    inner slab plane (the owned part may then differ from the whole
                                    grid's); 0 with whole-grid flips */
} odc_slab_info;

/* Extract one slab of ``grid`` (same source, parameters and stream rules
 * as odc_extract; ODC_POLY_MC is not supported).  ``out`` is the slab
 * extraction's own mesh (context memory, valid until the next extract on
 * this context); ``info`` locates its owned part.  Grid limits: res[0],
 * res[1] <= 2048, res[2] <= 8192, and the slab with its halo must keep
 * 3 (res[0]+1)(res[1]+1)(layers+1) below 2^32.  ODC_ERR_INVALID_ARG
 * otherwise. */
odc_status odc_extract_slab(odc_ctx* ctx, const odc_source* src, const odc_grid* grid, const odc_params* params,
                            const odc_slab* slab, void* cuda_stream, odc_mesh* out, odc_slab_info* info);

/* Label words of the vertex layers [z0, z1] of ``grid`` (the grid stage of
 * the path on that window) into d_bits, the whole grid's label words
 * (device, caller-owned, layout above); layers outside are not touched.
 * Synchronous. */
odc_status odc_grid_labels(odc_ctx* ctx, const odc_source* src, const odc_grid* grid, const odc_params* params,
                           int32_t z0, int32_t z1, uint32_t* d_bits, void* cuda_stream);

/* The manifold fix (A.1.1) of the whole grid from its complete label words:
 * the ambiguous faces are gathered in ``n_chunks`` windows of layers, then
 * rounds of mark-all / flip-all run over all of them; d_flips (device,
 * caller-owned) receives the flip words.  *n_flips = faces flipped.
 * Synchronous. */
odc_status odc_manifold_flips(odc_ctx* ctx, const odc_grid* grid, const uint32_t* d_bits, uint32_t* d_flips,
                              int32_t n_chunks, void* cuda_stream, int64_t* n_flips);

/* Place the owned part of a slab extraction (``mesh``, ``info`` from
 * odc_extract_slab on this context, before any other extract) into the
 * whole grid's mesh in device memory: 3D points at vertex index
 * ``verts3_base`` (the owned 3D points of all slabs below), edge points at
 * vertex index ``case3_base`` (all slabs' 3D points plus the owned edge
 * points of the slabs below), triangles at ``tris_base``.  d_verts
 * float[3 * total vertices], d_tris int32[3 * total triangles], device
 * pointers owned by the caller.  Asynchronous on ``cuda_stream``. */
odc_status odc_slab_place(odc_ctx* ctx, const odc_mesh* mesh, const odc_slab_info* info, int64_t verts3_base,
                          int64_t case3_base, int64_t tris_base, float* d_verts, int32_t* d_tris,
                          void* cuda_stream);

/* The whole grid in ``n_slabs`` slabs of near-equal depth, one after the
 * other on this context (peak device memory: one slab's arenas plus the
 * whole grid's label and flip words), the manifold fix taken from the
 * whole grid, merged into one mesh in context memory (valid until the next
 * extract).  The result equals
 * odc_extract's mesh on the same grid byte for byte; stats are summed over
 * the slabs (element counts include halo layers).  Grid limits as for
 * odc_extract_slab. */
odc_status odc_extract_slabbed(odc_ctx* ctx, const odc_source* src, const odc_grid* grid, const odc_params* params,
                               int32_t n_slabs, int32_t halo, void* cuda_stream, odc_mesh* out);

/* Upload an occupancy source (host descriptors) to the context's device
 * memory without extracting, so that later odc_extract calls with kind
 * ODC_SRC_RESIDENT start from device-resident inputs.  Returns
 * ODC_ERR_INVALID_ARG for a malformed source. */
odc_status odc_source_upload(odc_ctx* ctx, const odc_source* src);

/* Copy a mesh into caller buffers: verts float[n_verts*3], tris
 * int32[n_tris*3]; ``dst_on_device`` selects device or host destinations.
 * Synchronous.  Either pointer may be NULL to skip it. */
odc_status odc_mesh_copy(odc_ctx* ctx, const odc_mesh* mesh, float* verts, int32_t* tris,
                         int dst_on_device);

/* Mark the mesh's memory reusable (the next extract reuses it anyway). */
odc_status odc_mesh_release(odc_ctx* ctx, odc_mesh* mesh);

/* Intermediate buffers of the last extract, for parity checks.  Copies at
 * most ``max_bytes`` of buffer ``what`` into host memory ``dst`` and stores
 * the element count in *count and the element size in *elem_bytes:
 *   ODC_DBG_LABELS     uint32 label bit rows [res2+1][res1+1][ceil((res0+1)/32)]
 *   ODC_DBG_EDGES      uint32 crossing edge ids (sorted)
 *   ODC_DBG_T          uint32 1D results T (odd; point = T / 2^(k+1) along the edge)
 *   ODC_DBG_FACES      uint32 face ids of the 2D points (sorted with slots)
 *   ODC_DBG_SLOTS      uint8 segment slot of each 2D point
 *   ODC_DBG_FACE_PTS   float4 face-local 2D point as float-float pairs
 *                      (u_hi, u_lo, v_hi, v_lo): u = u_hi + u_lo
 *   ODC_DBG_FACE_FLAGS uint8 bit0: q == m, bit1: parallel lines
 *   ODC_DBG_CELLS      uint32 crossing cell ids (sorted)
 *   ODC_DBG_CONFIGS    uint8 cell configurations
 *   ODC_DBG_CYCLES     uint64 per cell: 4-bit cycle index per local edge (0xF: none)
 *   ODC_DBG_VLOCAL     float3 cell-local 3D points
 *   ODC_DBG_QCASE      uint8 per crossing edge: 0 no quad, 1/2/3 split case
 *   ODC_DBG_FLIPS      uint32 ids of faces flipped by the manifold fix (sorted)
 *   ODC_DBG_SEARCH     16 bytes per 2D point: uint32 Jq, J1, J2 (near-end
 *                      parameters of the three line-binary searches, sample
 *                      s = R J / (N 2^b)), uint8 label of m, uint8 found
 *                      (bit0 step 1, bit1 ray r1, bit2 ray r2 met a label
 *                      change in their linear phase), 2 pad bytes
 */
enum { ODC_DBG_LABELS = 0, ODC_DBG_EDGES, ODC_DBG_T, ODC_DBG_FACES, ODC_DBG_SLOTS,
       ODC_DBG_FACE_PTS, ODC_DBG_FACE_FLAGS, ODC_DBG_CELLS, ODC_DBG_CONFIGS,
       ODC_DBG_CYCLES, ODC_DBG_VLOCAL, ODC_DBG_QCASE, ODC_DBG_FLIPS, ODC_DBG_SEARCH, ODC_DBG_COUNT };
odc_status odc_debug_copy(odc_ctx* ctx, int what, void* dst, size_t max_bytes,
                          int64_t* count, int32_t* elem_bytes);

/* Evaluate the occupancy of ``src`` at n points (host float[n][3]) on the
 * device and return labels (host uint8[n]) and, for MLP sources, logits
 * (host float[n], may be NULL).  ``precision`` overrides the MLP precision
 * (-1 keeps the source's).  Sec. 3 / A.2.2 binary occupancy. */
odc_status odc_eval_points(odc_ctx* ctx, const odc_source* src, const float* points, int64_t n,
                           float iso, int precision, uint8_t* labels, float* logits);

/* Mesh quality: the measures of the paper's evaluation (Sec. 6.1 "Evaluation
 * Metrics") for a mesh in device memory (an odc_extract or odc_poll result).
 *   ODC_Q_OCC: |phi - iso| at n_samples points drawn uniformly by area on the
 *     mesh (counter-based SplitMix64 from ``seed``), phi = sigmoid of the FP32
 *     logit of the context's resident MLP source (the source of its last
 *     extract).  A CSG source's occupancy is binary; its fidelity is the
 *     first-order distance |psi| / |grad psi| of the implicit psi (the min/max
 *     fold of the primitives' g, FP64) at the same samples.
 *   ODC_Q_MANIFOLD: every directed edge used once with its reverse used once,
 *     every vertex fan a single cycle; Euler characteristic V - E + F.
 *   ODC_Q_SI: triangle pairs that intersect: pairs sharing no vertex whose
 *     closed sets meet, or sharing one vertex where the edge of either
 *     opposite to it meets the other; pairs sharing an edge never count.
 * Scratch is allocated on the context's stream and freed before return. */
enum { ODC_Q_OCC = 1, ODC_Q_MANIFOLD = 2, ODC_Q_SI = 4 };

typedef struct {
    int64_t n_samples;
    double occ_dev_mean;         /* MLP source: mean |phi - iso| over the samples; CSG: NaN */
    double occ_dev_max;
    double dist_mean;            /* CSG source: mean first-order distance |psi| / |grad psi|; MLP: NaN */
    double dist_max;
    int64_t n_tris;
    int64_t n_verts;             /* vertices used by a triangle */
    int64_t n_edges;             /* undirected edges */
    int64_t euler;               /* V - E + F */
    int64_t n_degenerate;        /* triangles with a repeated vertex */
    int64_t n_bad_edges;         /* directed edge uses not matched one-to-one by the reverse edge */
    int64_t n_bad_verts;         /* vertices whose fan is not a single cycle */
    int32_t manifold;            /* 1: closed, oriented 2-manifold */
    int32_t si_checked;
    int64_t n_si_pairs;          /* intersecting triangle pairs */
    int64_t n_si_tris;           /* triangles in at least one such pair */
} odc_quality;

odc_status odc_mesh_quality(odc_ctx* ctx, const odc_mesh* mesh, float iso, int64_t n_samples, uint64_t seed,
                            int32_t what, odc_quality* out);

/* ---- Request loop ---------------------------------------------------------
 * A server meshes requests of any grid size as they arrive.  Up to ``slots``
 * requests are on the GPU at once, each on its own stream with its own
 * context (device arenas, network weights), so their kernels and host round
 * trips overlap on the device.  Requests are admitted in arrival order when a
 * slot is free and the estimated device memory of the admitted requests plus
 * the results not yet released stays within ``mem_budget``.  Each request runs
 * exactly the odc_extract path, so its mesh is byte-identical whether it runs
 * alone or among others.  The paper meshes one shape per call (Sec. 3); the
 * loop is this library's serving layer around that call. */
typedef struct odc_server odc_server;

typedef struct {
    int32_t device;
    int32_t slots;               /* requests on the GPU at once, 1..64 */
    size_t mem_budget;           /* bytes over admitted requests and held results; 0 = no limit */
    int32_t host_copy;           /* nonzero: results also carry host copies of the mesh */
    int32_t share_network;       /* nonzero: the slots' contexts form one batch group, so requests in
                                    their search stages at the same time share network launches */
} odc_server_config;

typedef struct {
    odc_status status;           /* the request's own result (ODC_OK or its error) */
    int32_t slot;                /* slot that ran it */
    odc_mesh mesh;               /* device buffers owned by the server until odc_result_release */
    const float* h_verts;        /* host copies when host_copy is set (same lifetime), else NULL */
    const int32_t* h_tris;
    double t_submit, t_start, t_end;   /* seconds on the server's monotonic clock */
    uint64_t est_bytes;          /* device memory charged to the request at admission */
} odc_result;

/* Create a server (one context and one worker thread per slot). */
odc_status odc_server_create(const odc_server_config* cfg, odc_server** out);
/* Finish every queued and admitted request, then free everything, including
 * unreleased results.  NULL is accepted. */
odc_status odc_server_destroy(odc_server* srv);
/* Queue one request.  The source (primitives or weights and latent), grid and
 * parameters are copied: the caller may reuse its buffers at once.
 * ODC_SRC_RESIDENT is rejected (ODC_ERR_INVALID_ARG), as are arguments
 * odc_extract would reject.  *req_id identifies the request. */
odc_status odc_submit(odc_server* srv, const odc_source* src, const odc_grid* grid, const odc_params* prm,
                      uint64_t* req_id);
/* Wait up to timeout_ms milliseconds (negative: no limit) for a request.
 * ODC_ERR_TIMEOUT: not finished yet; ODC_ERR_INVALID_ARG: unknown id.
 * Otherwise *out describes the finished request (its own status inside). */
odc_status odc_poll(odc_server* srv, uint64_t req_id, int32_t timeout_ms, odc_result* out);
/* Free a finished request's result buffers and forget the request. */
odc_status odc_result_release(odc_server* srv, uint64_t req_id);
/* Seconds on the server's monotonic clock (the time base of odc_result). */
double odc_server_clock(const odc_server* srv);

/* ---- Shared network evaluations (batch groups) ------------------------------
 * The paper evaluates its network once per search step over all active
 * edges or faces of one shape (Sec. 5.1, 5.2).  Contexts that join a batch
 * group share those evaluations across shapes: inside a search stage each
 * network evaluation waits until every context currently in a search stage
 * of the group has made one, then all of their queries go through one
 * merged evaluation (one set of tensor-core and FP32 launches) on the
 * group's stream, and each context's stream waits for it.  Members must
 * share one network (the same B, W and b; latents may differ: each shape's
 * latent, folded into its first-layer bias, travels with its queries) and
 * one precision; others evaluate on their own.  Every mesh is byte-identical
 * to the one odc_extract gives without the group.  The grid pass is not
 * shared (it is one large evaluation per shape already).  A group holds at
 * most 64 members' bias rows.  Network statistics of members' extractions
 * then cover their own launches only. */
typedef struct odc_batch odc_batch;

/* Create / destroy a group on a device.  Destroy after its members have left
 * it (odc_ctx_join_batch(ctx, NULL)) or been destroyed. */
odc_status odc_batch_create(int device, odc_batch** out);
odc_status odc_batch_destroy(odc_batch* b);

/* Join a context to group b (NULL: leave).  Binding happens at the
 * context's next MLP source upload (odc_extract with an MLP source, or
 * odc_source_upload).  A member's shared evaluation waits on the host until
 * every member inside a search stage has made its call; a call that no
 * round takes within 120 s fails with ODC_ERR_TIMEOUT, and so does that
 * member's odc_extract. */
odc_status odc_ctx_join_batch(odc_ctx* ctx, odc_batch* b);

/* Merged evaluation rounds run by the group and the member calls they
 * served (calls / rounds is the mean number of shapes per launch). */
odc_status odc_batch_stats(const odc_batch* b, int64_t* rounds, int64_t* calls);

/* Extract n shapes at once, one host thread per context (all distinct), the
 * contexts joined to group b (NULL: no sharing).  outs[i] and statuses[i]
 * are shape i's odc_extract result; returns the first failing status. */
odc_status odc_extract_many(odc_batch* b, int32_t n, odc_ctx* const* ctxs, const odc_source* srcs,
                            const odc_grid* grids, const odc_params* prms, odc_mesh* outs, odc_status* statuses);

/* List the crossing edges of a label bitmask without allocating any memory.
 * The paper has no counterpart: this serves callers that cannot call
 * cudaMalloc (inside a stream capture that must not gain allocation nodes,
 * allocator-free hosts, plug-ins whose host owns all device memory).  It
 * computes what the compaction stage of odc_extract computes for edges.
 *   d_label_bits: device, uint32 label rows [res2+1][res1+1][ceil((res0+1)/32)]
 *                 as returned for ODC_DBG_LABELS (bit x of word x/32 = vertex x).
 *   res:          host, cells per axis (1..1024); the grid may hold at most
 *                 520,000 label words (e.g. 240^3 cells: 464,648 words).
 *   d_edges:      device, caller-owned, room for max_edges uint32 edge ids
 *                 (3 v + a, ascending); ids beyond max_edges are not written.
 *   d_count:      device uint32, receives the number of crossing edges.
 *   h_count:      optional host uint32; when given, the call synchronises the
 *                 stream, stores the count and returns ODC_ERR_OOM if it
 *                 exceeds max_edges.
 *   cuda_stream:  cudaStream_t (NULL: the legacy default stream).
 * Scratch lives in a 4 MiB file-scope device array that every GPU loading
 * the library keeps until exit.  The first call on each device looks up its
 * address (make that first call before any stream capture).  All calls on a
 * device share the array: calls that overlap on the GPU race.  Grids above
 * the limit return ODC_ERR_INVALID_ARG; nothing is allocated on any path. */
odc_status odc_compact_edges_noalloc(const uint32_t* d_label_bits, const int32_t res[3], uint32_t* d_edges,
                                     uint32_t max_edges, uint32_t* d_count, uint32_t* h_count,
                                     void* cuda_stream);

/* Number of CUDA kernel launches the library has issued since it was loaded
 * (all contexts and threads); lets a caller count the kernels of a region. */
int64_t odc_launch_count(void);

const char* odc_status_str(odc_status s);
const char* odc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ODC_H */
