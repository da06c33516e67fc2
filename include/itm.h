/*
 * itm.h -- C ABI of the GB300 hashed-TSDF library (libitm.so).
 *
 * The library implements the per-frame data-parallel core of voxel-hashing
 * reconstruction described in InfiniTAM v3 (Prisacariu et al., 2017):
 * allocation of voxel blocks into a spatial hash (Sec. 4.2, hash structure of
 * Sec. 3.2-3.3), TSDF/weight integration over the visible blocks (Sec. 4.3)
 * and raycasting the volume into vertex and normal maps (Sec. 4.4).
 *
 * Conventions shared by every call:
 *  - Camera frame: +x right, +y down, +z forward; u = fx*X/Z + cx,
 *    v = fy*Y/Z + cy; pixel (u, v) is column u, row v.
 *  - A pose T_wc is a rigid camera-to-world 4x4 matrix, float[16], row-major,
 *    passed as a HOST pointer and read before the call returns.  The library
 *    forms M_d = T_wc^-1 on the host in double precision as [R^T, -R^T t] and
 *    rounds it to float.
 *  - Depth images are float32 metres, row-major [height][width], 0 (or any
 *    value that is not > 0) = no measurement, held in DEVICE memory owned by
 *    the caller.
 *  - Output images are DEVICE memory owned by the caller.
 *  - Every compute call is asynchronous on the given stream (a cudaStream_t
 *    passed as itm_stream; NULL is the legacy default stream).  Kernel-side
 *    errors (hash or block array exhausted, coordinate out of range, a bounded
 *    wait that gave up) set bits in a sticky device status word that is read
 *    by itm_scene_stats / itm_scene_status, which synchronise the stream.
 *  - A scene owns all of its device memory; no call after itm_scene_create
 *    allocates device memory.  Calls on one scene must not overlap in time
 *    (not thread-safe per scene); different scenes are independent.
 *  - Return value: ITM_OK or one of the ITM_ERR_* codes below.  A call that
 *    returns an error has launched nothing.
 */
#ifndef ITM_H
#define ITM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void *itm_stream; /* a cudaStream_t */

enum {
    ITM_OK = 0,
    ITM_ERR_ARG = 1,       /* invalid argument (null pointer, bad size, bad parameter) */
    ITM_ERR_CUDA = 2,      /* a CUDA runtime call failed */
    ITM_ERR_HASH_FULL = 3, /* status: excess list exhausted */
    ITM_ERR_VBA_FULL = 4,  /* status: voxel block array exhausted */
    ITM_ERR_RANGE = 5,     /* status: block coordinate outside int16 */
    ITM_ERR_TIMEOUT = 6,   /* status: a bounded device-side wait gave up */
    ITM_ERR_OVERFLOW = 7,  /* status: a per-frame work list overflowed */
    ITM_ERR_TOO_LARGE = 8, /* the input could exceed a fixed-size buffer of the call */
    ITM_ERR_SINGULAR = 9,  /* a tracking step has no unique solution (fewer than 6 constrained motions) */
    ITM_ERR_BOUNDS = 10,   /* status: an index check failed (bounds-checked builds; the swap kernels always) */
};

/* Sticky status bits (itm_stats.status). */
#define ITM_ST_HASH_FULL 0x1u
#define ITM_ST_VBA_FULL 0x2u
#define ITM_ST_RANGE 0x4u
#define ITM_ST_TIMEOUT 0x8u
#define ITM_ST_OVERFLOW 0x10u
#define ITM_ST_BOUNDS 0x20u /* an index was out of range, the access skipped: in builds with -DITM_CHECK_BOUNDS,
                              * and in every build for a swap entry that is not what its selection said */

/* Pinhole depth intrinsics (Sec. 6 calibration file: image size, focal
 * length and principal point in pixels; Sec. 4.3 projParams_d). */
typedef struct {
    int width, height;
    float fx, fy, cx, cy;
} itm_intrinsics;

/* Scene parameters (Sec. 6 ITMSceneParams; Sec. 3.1 voxel block array size;
 * Sec. 3.2 bucket count; Sec. 4.3 mu and maxW).
 *  voxel_size  metres per voxel (s); a block is 8 voxels per axis
 *  mu          truncation band (metres), 2^-64 <= mu < 2^64
 *  max_w       weight cap; 1..255 in weight_mode 0
 *  num_buckets ordered part of the hash table, a power of two
 *  num_excess  unordered excess entries
 *  num_blocks  voxel blocks in the block array
 *  z_min/z_max depth range for allocation and for the raycast march
 *  weight_mode 0: constant observation weight 1, uint8 weights (Sec. 4.3);
 *              1: per-pixel observation weight from itm_integrate_weighted,
 *                 float32 weights */
typedef struct {
    float voxel_size, mu;
    int max_w;
    int num_buckets, num_excess, num_blocks;
    float z_min, z_max;
    int weight_mode;
} itm_scene_params;

/* Counters kept on the device, cumulative since the last reset unless noted. */
typedef struct {
    uint32_t status;            /* sticky ITM_ST_* bits */
    int32_t allocated_blocks;   /* blocks handed out from the block array */
    int32_t excess_used;        /* excess entries handed out */
    int32_t visible_blocks;     /* blocks in the last frame's visible list */
    int32_t last_requests;      /* new blocks requested by the last allocation */
    int32_t last_overflow;      /* requests that lost a bucket in the last allocation */
    uint64_t updated_voxels;    /* voxel updates performed by integration */
    uint64_t visited_voxels;    /* voxels visited by integration (512 per visible block) */
    uint64_t frames;            /* completed itm_integrate calls */
} itm_stats;

typedef struct itm_scene itm_scene;

/* Create a scene on the current CUDA device: allocates the hash table
 * ((num_buckets + num_excess) entries of 16 bytes: int16 x, y, z, a flag,
 * int32 offset, int32 ptr; Sec. 3.2), the voxel block array (Sec. 3.1: per
 * block 512 float sdf + 512 weights), the free lists (Sec. 3.3) and the
 * per-frame work lists, then resets it and synchronises.  *out receives the
 * handle.  Errors: ITM_ERR_ARG for invalid parameters, ITM_ERR_CUDA if
 * device memory cannot be allocated (nothing is leaked). */
int itm_scene_create(const itm_scene_params *params, itm_scene **out);

/* Release all device memory of the scene (synchronises the device). */
int itm_scene_destroy(itm_scene *scene);

/* Empty the scene: every entry unallocated (ptr = -2, offset 0), every voxel
 * sdf = 1, weight = 0 (Sec. 3.1 defaults), full free lists, counters and
 * status cleared.  Asynchronous on `stream`. */
int itm_scene_reset(itm_scene *scene, itm_stream stream);

/* Sec. 4.2 allocation.  For each pixel with z_min <= d <= z_max, the blocks
 * crossed by the segment of the pixel's ray between z-depth d - mu and
 * d + mu are looked up (Sec. 3.3 retrieval) and every missing one is
 * inserted (Sec. 3.3 insertion), including blocks that collide in one hash
 * bucket within the frame.  Then the visible list is rebuilt: every
 * allocated block whose voxels may project into the image with z > 0 and lie
 * no further than the frame's largest depth + mu.
 * depth_dev: device float[height*width].  intr, T_wc: host pointers. */
int itm_allocate(itm_scene *scene, const float *depth_dev, const itm_intrinsics *intr,
                 const float T_wc[16], itm_stream stream);

/* Sec. 4.3 integration over the visible list built by the last
 * itm_allocate: for every voxel, project with M_d = T_wc^-1, skip unless
 * z > 0, 1 <= u <= W-2, 1 <= v <= H-2, the nearest pixel's depth d > 0 and
 * eta = d - z >= -mu; then F <- (W F + min(1, eta/mu)) / (W + 1),
 * W <- min(W + 1, max_w).  Must use the same depth and pose as the
 * preceding itm_allocate. */
int itm_integrate(itm_scene *scene, const float *depth_dev, const itm_intrinsics *intr,
                  const float T_wc[16], itm_stream stream);

/* As itm_integrate, with a per-pixel observation weight w_px (device
 * float[height*width]) in place of the constant 1: F <- (W F + w_px f) /
 * (W + w_px), W <- min(W + w_px, max_w); pixels with w_px <= 0 are skipped.
 * Requires weight_mode 1. */
int itm_integrate_weighted(itm_scene *scene, const float *depth_dev, const float *wpx_dev,
                           const itm_intrinsics *intr, const float T_wc[16], itm_stream stream);

/* Sec. 4.4 raycast.  One ray per pixel from the camera centre, marched from
 * z-depth z_min to z_max through the states SEARCH_BLOCK_COARSE (block-sized
 * steps through unallocated space), SEARCH_BLOCK_FINE (steps of mu after
 * stepping back one block), SEARCH_SURFACE (steps of max(F mu, s)) and
 * BEHIND_SURFACE (first F <= 0), or WRONG_SIDE (negative F on entering a
 * block: no hit); the hit is refined by two trilinear steps t += F mu.
 * vertex_dev: device float4[height*width], world (x, y, z, 1) or 0 on a miss.
 * normal_dev: device float4[height*width], the normalised TSDF gradient by
 * central differences (x, y, z, 1), or 0 when absent. */
int itm_raycast(itm_scene *scene, const itm_intrinsics *intr, const float T_wc[16],
                float *vertex_dev, float *normal_dev, itm_stream stream);

/* Sec. 4.4 search range, per 8x4-pixel tile (tile (i, j) covers pixels
 * u = 8i .. 8i+7, v = 4j .. 4j+3; ceil(width/8) x ceil(height/4) tiles,
 * row-major): the nearest and farthest camera depth of the allocated blocks
 * that can cover the tile, each block taken as the region of points whose
 * nearest voxel it holds, clipped to z >= z_min, with small margins.  A tile
 * no block covers gets zmin = NaN (all bits set) and zmax = 0.  zmin_dev,
 * zmax_dev: device float[tiles].  itm_raycast computes the same range
 * internally (for images up to 4096 x 4096) and uses it only to skip hash
 * probes it can prove unallocated; its result does not depend on it. */
int itm_raycast_range(itm_scene *scene, const itm_intrinsics *intr, const float T_wc[16], float *zmin_dev,
                      float *zmax_dev, itm_stream stream);

/* Sec. 7.2 combined map: raycast of the global map formed by n posed
 * submaps (1 <= n <= ITM_COMBINED_MAX), rendered as a view over them without
 * building it.  At a world point X the combined TSDF is
 *   sum_i W_i(P_i X) F_i(P_i X) / sum_i W_i(P_i X)
 * with F_i and W_i the trilinearly interpolated TSDF and weight of submap i
 * (an unallocated voxel counts as F = 1, W = 0), summed in index order, and
 * 1 where the weight sum is 0.  (The paper prints the sum without the
 * division; dividing by the positive weight sum keeps its zero set and gives
 * the raycast's step rule a value in [-1, 1].)  The march, refinement and
 * outputs are those of itm_raycast in world coordinates, "allocated" meaning
 * that the block of the voxel nearest to P_i X is allocated in some submap;
 * the normal is the normalised central difference of the combined value at
 * X +- voxel_size along each world axis, absent (0) when one of the six
 * samples has weight 0 in every submap.
 * scenes: host array of n scene handles; all must share voxel_size, mu,
 * z_min, z_max and weight_mode (else ITM_ERR_ARG).  submap_from_world: host
 * float[n][16], row-major rigid transforms P_i mapping world coordinates to
 * submap i's coordinates (the submap's own frame, in which it was fused).
 * T_wc, vertex_dev, normal_dev: as for itm_raycast (world frame).  The scenes
 * are only read; the call allocates nothing; asynchronous on stream. */
#define ITM_COMBINED_MAX 16
int itm_raycast_combined(itm_scene *const *scenes, const float *submap_from_world, int n,
                         const itm_intrinsics *intr, const float T_wc[16], float *vertex_dev, float *normal_dev,
                         itm_stream stream);

/* ---------------------------------------------------------------------
 * One scene split over several processes (one per GPU) by slabs of block
 * columns.  The paper has no counterpart: it is the multi-process form of
 * the per-frame core of Sec. 4.2-4.4.  Block column x belongs to part
 * floor(x / slab_blocks) mod parts.  A part allocates and integrates the
 * blocks of its own columns and of one column on either side (every sample
 * the raycast takes around a point of its own columns reads the same voxels
 * as in the whole scene; those voxels are bit-identical to the whole
 * scene's), so every process receives the whole depth frame and no data
 * moves between processes until the raycast.  Each part's raycast reports
 * only hits in its own columns; the parts' maps, gathered on every process,
 * merge per pixel to the hit nearest to the camera (itm_raycast_merge).  The
 * merged map is close to the whole scene's, not identical: a ray that
 * reaches a part's columns from space the part does not hold starts its fine
 * search there, so near slab boundaries a refined hit can move by a few mm.
 */

/* Make the scene part `index` of `parts` (1 <= parts, 0 <= index < parts,
 * slab_blocks >= 2 block columns per slab); parts = 1 restores the whole
 * scene.  Applies to later allocations and raycasts (blocks allocated before
 * stay).  Host only.  Errors: ITM_ERR_ARG for invalid values. */
int itm_scene_set_shard(itm_scene *scene, int parts, int index, int slab_blocks);

/* Merge the raycasts of the parts of a split scene: vertex_parts_dev and
 * normal_parts_dev hold `parts` maps of width x height float4, one part
 * after another (as an all-gather leaves them); per pixel the hit (w = 1)
 * with the smallest camera depth (row 2 of the world-to-camera transform,
 * formed from T_wc as for itm_raycast, applied to the vertex with each
 * operation rounded on its own) is copied to vertex_dev / normal_dev, equal
 * depths going to the lower part; pixels with no hit get zeros.  All
 * buffers are caller device memory, 16-byte aligned.  Asynchronous on
 * `stream`.  Errors: ITM_ERR_ARG for null or unaligned buffers, parts < 1,
 * invalid intrinsics or pose. */
int itm_raycast_merge(const float *vertex_parts_dev, const float *normal_parts_dev, int parts,
                      const itm_intrinsics *intr, const float T_wc[16], float *vertex_dev, float *normal_dev,
                      itm_stream stream);

/* ---------------------------------------------------------------------
 * Sec. 4.1.1 depth tracker (ITMDepthTracker): align a depth frame to the
 * vertex and normal maps of an itm_raycast by minimising the sum of squared
 * point-to-plane distances, over a resolution hierarchy of the depth image.
 */

/* One level of the depth pyramid: out_dev[j][i] (floor(width/2) x
 * floor(height/2), device float) is the mean of the valid (> 0) depths of
 * in_dev's pixels (2i, 2j), (2i+1, 2j), (2i, 2j+1), (2i+1, 2j+1), summed in
 * that order and divided once by their count; 0 when none is valid.  The
 * level's intrinsics are fx/2, fy/2, (cx - 1/2)/2, (cy - 1/2)/2. */
int itm_depth_halve(const float *in_dev, int width, int height, float *out_dev, itm_stream stream);

#define ITM_ICP_SUMS 29
#define ITM_ICP_WORK_DOUBLES (ITM_ICP_SUMS * 1025)

/* One evaluation of the tracker's linear system.  For each pixel of
 * depth_dev (device float[height][width] of intr) with depth d > 0, the
 * camera point d ((u-cx)/fx, (v-cy)/fy, 1) is mapped to the world by the
 * estimate T_g (camera-to-world) and projected into the reference view
 * (pose T_ref, intrinsics ref_intr) of the maps vertex_dev / normal_dev
 * (device float4[ref height][ref width], world coordinates, w > 0 valid, as
 * written by itm_raycast); at the nearest pixel, when both maps are valid and
 * |T_g p - V| <= dist_thresh, the residual r = (T_g p - V) . N and its
 * derivative J = (T_g p x N, N) with respect to a small world-frame motion
 * (rotation omega, translation tau) enter the sums.  Per-pixel arithmetic
 * is float with every operation rounded on its own; a thread sums its pixels
 * in float, the rest of the reduction is double, in a fixed order.
 * work_dev: device double[ITM_ICP_WORK_DOUBLES] (8-byte aligned); on return
 * (asynchronous) work_dev[0..28] hold sum J_i J_j (i <= j, row-major upper
 * triangle, 21), sum J_i r (6), sum r^2 and the number of pixels used. */
int itm_icp_reduce(const float *depth_dev, const itm_intrinsics *intr, const float T_g[16],
                   const float *vertex_dev, const float *normal_dev, const itm_intrinsics *ref_intr,
                   const float T_ref[16], float dist_thresh, double *work_dev, itm_stream stream);

/* Host: one Gauss-Newton step from the sums (HOST double[29], as written by
 * itm_icp_reduce): solve H x = -g by Cholesky in double and apply the motion
 * x = (omega, tau) on the world side, T <- [R(omega) | tau] T (Rodrigues).
 * T_inout: host float[16]; step_out (nullable): host double[6].  Returns
 * ITM_ERR_SINGULAR (T unchanged) when fewer than 6 pixels were used or H is
 * not positive definite. */
int itm_icp_step(const double *sums, float T_inout[16], double *step_out);

#define ITM_TRACK_MAX_LEVELS 8

/* Bytes of device scratch itm_track_depth needs for an image of width x
 * height and the given number of levels. */
size_t itm_track_scratch_bytes(int width, int height, int levels);

/* Coarse-to-fine tracking of one depth frame (device float[height][width]
 * of intr) against the maps of a raycast from T_ref: pyramid levels
 * 0 (input) .. levels-1 (1 <= levels <= ITM_TRACK_MAX_LEVELS); from the
 * coarsest level down, iters[l] steps (itm_icp_reduce + the step of
 * itm_icp_step, taken on the device in double) with outlier distance
 * dist_thresh[l] (host arrays of levels entries); a level ends early when a
 * step has no unique solution.  T_inout: host float[16], the initial
 * camera-to-world estimate, replaced by the result; steps_out (nullable):
 * the steps applied.  scratch_dev: device memory of
 * itm_track_scratch_bytes(width, height, levels) bytes, 256-byte aligned,
 * owned by the caller, contents irrelevant.  Synchronises the stream once at
 * the end (no host round trip per step). */
int itm_track_depth(const float *depth_dev, const itm_intrinsics *intr, int levels, const int *iters,
                    const float *dist_thresh, const float *vertex_dev, const float *normal_dev,
                    const itm_intrinsics *ref_intr, const float T_ref[16], float T_inout[16], int *steps_out,
                    void *scratch_dev, itm_stream stream);

/* Sec. 4 mesh generation by Marching Cubes (Lorensen & Cline 1987): the
 * zero level set of the TSDF (inside: F < 0) over every cell g + {0,1}^3
 * whose eight corner voxels are allocated and observed (weight > 0).  The
 * triangulation of each corner pattern comes from walking the cube's faces
 * (a face with two diagonal inside corners cuts off each of them, so cells
 * sharing a face agree and the mesh is closed); each crossing loop is fanned
 * from its crossing on the lowest-numbered edge, triangles counter-clockwise
 * seen from outside (F > 0).  A vertex on the edge from voxel g_a to g_b
 * (one axis step up) sits at (g_a + t) s along that axis, t = F_a / (F_a -
 * F_b).  triangles_dev: device float[capacity][9] (three world-space
 * vertices per triangle; order of triangles unspecified), may be NULL when
 * capacity is 0.  *n_out (host): the number of triangles in the mesh.
 * Returns ITM_ERR_TOO_LARGE when that exceeds capacity (capacity of them
 * are written).  Synchronises the stream. */
int itm_mesh(itm_scene *scene, float *triangles_dev, int64_t capacity, int64_t *n_out, itm_stream stream);

/* The Marching-Cubes case table itm_mesh uses (Sec. 4 meshing), for
 * inspection: for each of the 256 inside/outside patterns of a cell's corners
 * (bit k set: corner k, at (k & 1, (k >> 1) & 1, k >> 2), has F < 0) count[cfg]
 * triangles, whose corners are the crossings on cube edges edges[15 * cfg +
 * 3 * t + 0..2], edge 4 a + o1 + 2 o2 running along axis a from the corner
 * whose other two coordinates are o1 (lower axis) and o2 (higher axis); each
 * triangle counter-clockwise seen from the F > 0 side.  count: host uint8[256],
 * edges: host uint8[256 * 15] (caller memory).  Host only, no device call.
 * Errors: ITM_ERR_ARG for a null pointer. */
int itm_mesh_case_table(uint8_t *count, uint8_t *edges);

/* itm_allocate on an unsigned short millimetre frame: the allocation reads
 * raw_dev (device uint16[height*width]) and converts each pixel as
 * itm_depth_u16_to_f32 does (raw / 1000, correctly rounded, Sec. 4 view
 * preparation), writing the float frame to depth_dev (device
 * float[height*width], caller-owned) for the integration that follows: one
 * pass over the frame instead of a separate conversion.  Same results as
 * itm_depth_u16_to_f32 followed by itm_allocate. */
int itm_allocate_u16(itm_scene *scene, const uint16_t *raw_dev, float *depth_dev, const itm_intrinsics *intr,
                     const float T_wc[16], itm_stream stream);

/* One frame from an unsigned short millimetre frame: itm_allocate_u16 (which
 * writes depth_dev), itm_integrate on depth_dev and (when vertex_dev is not
 * NULL) itm_raycast, on one stream. */
int itm_process_frame_u16(itm_scene *scene, const uint16_t *raw_dev, float *depth_dev, const itm_intrinsics *intr,
                          const float T_wc[16], float *vertex_dev, float *normal_dev, itm_stream stream);

/* One frame of the per-frame core: itm_allocate, itm_integrate and (when
 * vertex_dev is not NULL) itm_raycast, on one stream. */
int itm_process_frame(itm_scene *scene, const float *depth_dev, const itm_intrinsics *intr,
                      const float T_wc[16], float *vertex_dev, float *normal_dev,
                      itm_stream stream);

/* Sec. 4 view preparation: depth_dev[i] = raw_dev[i] / 1000 (millimetres
 * to metres, correctly rounded; 0 stays 0).  n elements, device memory. */
int itm_depth_u16_to_f32(const uint16_t *raw_dev, float *depth_dev, int64_t n, itm_stream stream);

/* Synchronise the scene's last stream and copy the device counters to
 * *out (host).  Returns ITM_OK, or ITM_ERR_CUDA. */
int itm_scene_stats(itm_scene *scene, itm_stats *out);

/* Synchronise and translate the sticky status into a return code:
 * ITM_OK when clear, else the code of the lowest set bit. */
int itm_scene_status(itm_scene *scene);

/* Copy the allocated blocks to HOST buffers (synchronises): coords_host
 * int16[cap][3] block coordinates, sdf_host float[cap][512] and w_host
 * float[cap][512] (either may be NULL), voxel index x + 8y + 64z, in block
 * array order.  *n receives the number of allocated blocks (which may
 * exceed cap; only min(n, cap) are written). */
int itm_scene_export(itm_scene *scene, int16_t *coords_host, float *sdf_host, float *w_host,
                     int cap, int *n);

/* Copy the raw hash table to a HOST buffer int32[num_buckets + num_excess][5]
 * (x, y, z, offset, ptr per entry; Sec. 3.2 field meaning).  Synchronises. */
int itm_scene_export_table(itm_scene *scene, int32_t *entries_host);

/* Reset the scene and insert n blocks from HOST buffers (coords int16[n][3],
 * sdf float[n][512], w float[n][512]); the inverse of itm_scene_export.
 * Duplicate coordinates or n > num_blocks give ITM_ERR_ARG.  Synchronises. */
int itm_scene_import(itm_scene *scene, const int16_t *coords_host, const float *sdf_host,
                     const float *w_host, int n);

/* The bucket of block (x, y, z) for a table of num_buckets buckets
 * (Sec. 3.2 hashIndex).  Host function, for tools and tests. */
uint32_t itm_hash_index(int x, int y, int z, int num_buckets);

/* ------------------------------------------------------------------------
 * Learned per-pixel confidence weight (not in the paper: it replaces the
 * constant observation weight 1 of the Sec. 4.3 listing through
 * itm_integrate_weighted).  Features of pixel (u, v): the 7x7 depth patch,
 * entry (i, j) at index (i+3)*7 + (j+3) = clamp((D(u+j, v+i) - D(u, v))/mu,
 * -4, 4) where that pixel is inside the image with depth > 0, else 0; then
 * the camera-facing unit normal of the back-projected depth from central
 * differences (0 when a neighbour is missing).  Network: h1 = relu(W1 x + b1),
 * h2 = relu(W2 h1 + b2) (64 each), w_px = sigmoid(w3 . h2 + b3); 0 for pixels
 * without depth.  Parameters: fp32, ITM_MLP_PARAMS values in the order
 * W1[64][52], b1[64], W2[64][64], b2[64], w3[64], b3.
 * ---------------------------------------------------------------------- */
#define ITM_MLP_FEATURES 52
#define ITM_MLP_HIDDEN 64
#define ITM_MLP_PARAMS 7617
/* packed inference weights: bf16 W1 (64 x 64, features zero-padded),
 * bf16 W2 (64 x 64), fp32 b1, b2, w3, b3 (+ 3 floats of padding) */
#define ITM_MLP_PACKED_BYTES 17168
/* training scratch, floats per sample */
#define ITM_MLP_SCRATCH_PER_SAMPLE 257

/* Round the fp32 parameters (device, ITM_MLP_PARAMS floats) into the packed
 * inference layout (device, ITM_MLP_PACKED_BYTES, 16-byte aligned): bf16
 * round-to-nearest-even for W1 and W2. */
int itm_mlp_pack(const float *params_dev, void *packed_dev, itm_stream stream);

/* w_px for every pixel of a depth frame (device float[height*width]) with
 * the packed network: features in fp32, both hidden layers as tcgen05
 * tensor-core products (bf16 operands, fp32 accumulators in tensor memory),
 * output layer in fp32.  Argument errors return ITM_ERR_ARG (packed_dev must
 * be 16-byte aligned).  Completion of each product is awaited with a bounded
 * wait; a wait that gives up (not expected on a healthy device) leaves NaN
 * weights in the tiles concerned, which itm_integrate_weighted skips. */
int itm_conf_weights(const float *depth_dev, const itm_intrinsics *intr, float mu, const void *packed_dev,
                     float *wpx_dev, itm_stream stream);

/* One frame of the per-frame core with the learned weight (Sec. 4.2-4.4,
 * the observation weight of the Sec. 4.3 listing replaced by w_px): the
 * per-pixel weights (itm_conf_weights, with the scene's mu, into wpx_dev)
 * run on the scene's second stream at the same time as the allocation on
 * `stream` (both read only the depth frame), then itm_integrate_weighted and,
 * with vertex_dev, itm_raycast on `stream`.  The results equal those of the
 * four calls in sequence.  The scene must be in weight_mode 1 (whose
 * itm_scene_create made the second stream and its events); wpx_dev is caller
 * device memory of width x height floats, written by the call.  Asynchronous
 * on `stream` (the second stream joins it before the integration).  Errors:
 * ITM_ERR_ARG for null buffers, another weight mode, invalid intrinsics or
 * pose; otherwise those of the four calls. */
int itm_process_frame_weighted(itm_scene *scene, const float *depth_dev, const void *packed_dev, float *wpx_dev,
                               const itm_intrinsics *intr, const float T_wc[16], float *vertex_dev,
                               float *normal_dev, itm_stream stream);

/* Features (device float[n][52]) of n pixels given by linear index
 * u + v * width (device int32[n]); out-of-range indices give zeros. */
int itm_conf_features(const float *depth_dev, const itm_intrinsics *intr, float mu, const int32_t *pixels_dev,
                      int n, float *feat_dev, itm_stream stream);

/* Mean binary cross-entropy of the network on n samples (features
 * float[n][52], labels float[n] in {0, 1}, device) into *loss_dev and its
 * gradient into grad_dev (ITM_MLP_PARAMS floats); the forward rounds W1, W2
 * and the layer inputs to bf16 exactly as itm_conf_weights does, and the
 * gradient treats that rounding as the identity.  scratch_dev: device float
 * [n][ITM_MLP_SCRATCH_PER_SAMPLE] owned by the caller. */
int itm_mlp_loss_grad(const float *params_dev, const float *feat_dev, const float *labels_dev, int n,
                      float *scratch_dev, float *grad_dev, float *loss_dev, itm_stream stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected for step
 * >= 1) on the fp32 parameters, with moments m_dev, v_dev (device,
 * ITM_MLP_PARAMS floats each, zero before step 1). */
int itm_mlp_adam(float *params_dev, const float *grad_dev, float *m_dev, float *v_dev, int step, float lr,
                 itm_stream stream);

/* ------------------------------------------------------------------------
 * Batches (InfiniTAM v3 Sec. 7.2 submaps; many independent scenes).  A batch
 * runs one frame for each of up to max_items (scene, frame) items through
 * allocation, integration and raycast with one launch per stage for the whole
 * batch; each scene gets exactly the arithmetic of itm_process_frame.  The
 * launches are persistent kernels whose sizes do not depend on the items, so
 * with a non-NULL stream they are captured into a CUDA graph on the first run
 * and replayed afterwards (itm_batch_set_graph(b, 0) turns this off).
 * ---------------------------------------------------------------------- */
typedef struct itm_batch itm_batch;

/* One item: a frame for one scene.  For a submap, T_wc is the camera pose in
 * that submap's frame (the world-to-submap transform times the camera's
 * world pose).  depth_dev may be shared by several items.  vertex_dev and
 * normal_dev (device float4[height*width], 16-byte aligned) receive the
 * raycast from T_wc; both NULL skips the raycast for the item. */
typedef struct {
    itm_scene *scene;
    const float *depth_dev;
    itm_intrinsics intr;
    float T_wc[16];
    float *vertex_dev;
    float *normal_dev;
} itm_batch_item;

/* Number of tunable batch stages: enumerate, commit, visible list,
 * integrate, search range, raycast. */
#define ITM_BATCH_STAGES 6

/* Create a batch for up to max_items (1..256) items on the current device:
 * device item table, pinned upload ring, default launch shapes.  Errors:
 * ITM_ERR_ARG, ITM_ERR_CUDA. */
int itm_batch_create(int max_items, itm_batch **out);
int itm_batch_destroy(itm_batch *batch);

/* Run one frame for each of the n items (host array, read before the call
 * returns).  All scenes must be distinct, in weight_mode 0, with images of
 * at most 4096 x 4096.  Asynchronous on `stream`; up to 4 runs may be in
 * flight before a call waits for the oldest upload. */
int itm_batch_run(itm_batch *batch, const itm_batch_item *items, int n, itm_stream stream);

/* CTAs per SM for each of the ITM_BATCH_STAGES persistent stages (0: as many
 * as fit); drops the captured graph.  itm_batch_get_tuning returns the grid
 * sizes in use. */
int itm_batch_set_tuning(itm_batch *batch, const int *ctas_per_sm, int n);
int itm_batch_get_tuning(itm_batch *batch, int *grid_ctas, int n);

/* The batch's schedule, ITM_BATCH_KNOBS values: [0] blocks one integration
 * CTA updates at once (1, 2 or 4; 64 threads each), [1] and [2] the
 * enumeration's and the raycast's walk over the virtual 32x8-pixel tiles of
 * all items (0: in item order; 1: scattered, tile v taken as v * P mod the
 * tile count for a P coprime to it, interleaving the items).  Results do not
 * depend on the schedule.  Drops the captured graph.  Default [1, 0, 0].
 * Errors: ITM_ERR_ARG for another count or value. */
#define ITM_BATCH_KNOBS 3
int itm_batch_set_schedule(itm_batch *batch, const int *knobs, int n);
int itm_batch_get_schedule(itm_batch *batch, int *knobs, int n);
int itm_batch_set_graph(itm_batch *batch, int use_graph);

/* Library version string. */
const char *itm_version(void);

/* Distinct blocks one itm_frame_blocks_noalloc call can hold. */
#define ITM_NOALLOC_MAX_BLOCKS (1 << 21)
/* Flag bits of itm_frame_blocks_noalloc's count (the low 30 bits count blocks). */
#define ITM_NOALLOC_RANGE 0x40000000
#define ITM_NOALLOC_OVERFLOW ((int32_t)0x80000000u)

/* The voxel blocks one depth frame touches, computed without allocating
 * memory.  The paper has no counterpart: this serves callers that cannot
 * call cudaMalloc once they are running -- a real-time loop that must not
 * wait on the allocator, a host framework whose device memory comes only
 * from its own fixed arenas, a system that forbids dynamic allocation after
 * start-up -- but want to know which blocks a frame needs (to reserve or
 * stream storage of their own).  It needs no scene.
 *
 * Result: the set of blocks that itm_allocate would insert into an empty
 * scene with these parameters (the segment d - mu .. d + mu of every pixel
 * with z_min <= d <= z_max, every block crossed), in no particular order, as
 * int16 (x, y, z) triples in coords_dev (caller device memory, cap triples);
 * *count_dev (caller device memory) receives in its low 30 bits the number of
 * distinct blocks, which may exceed cap (then only cap are written).  Bit 30
 * (ITM_NOALLOC_RANGE) is set when a pixel's segment left the int16 block
 * coordinates and the pixel was dropped (itm_allocate reports the same case
 * as ITM_ST_RANGE); bit 31 (a negative count, ITM_NOALLOC_OVERFLOW) when a
 * block found no slot in the fixed set within its probe limit (not expected
 * below the size check).
 *
 * Memory: the de-duplication set is a fixed device array of
 * 2 * ITM_NOALLOC_MAX_BLOCKS 64-bit words (32 MiB) inside the library,
 * present on every GPU that loads the library until the process exits.
 * The first call on a device looks up that array's address (with the
 * device current) and keeps it for the life of the process; make that first
 * call before any stream capture, and do not use the entry point across a
 * cudaDeviceReset.  Each
 * call clears the array and the count before use.  All calls share the
 * array: calls that overlap on the GPU (other streams, other host threads)
 * race and give wrong results.
 *
 * Errors: ITM_ERR_ARG for null pointers, invalid intrinsics, parameters, a
 * non-finite pose or one that is not rigid (last row 0 0 0 1, rotation rows
 * orthonormal within 1e-4); ITM_ERR_TOO_LARGE when width * height * (the most
 * blocks one pixel's segment can cross) exceeds ITM_NOALLOC_MAX_BLOCKS;
 * ITM_ERR_CUDA when a CUDA call fails.  Asynchronous on `stream`. */
int itm_frame_blocks_noalloc(const float *depth_dev, const itm_intrinsics *intr, const float T_wc[16],
                             float voxel_size, float mu, float z_min, float z_max, int16_t *coords_dev,
                             int cap, int32_t *count_dev, itm_stream stream);

/* ------------------------------------------------------------------------
 * Colour voxels (Sec. 3.1: the voxel types with colour carry an RGB value and
 * a colour weight; the paper does not print their update).  A voxel that gets
 * a depth update within the band -mu <= eta <= mu takes the colour of its
 * projection into the RGB image: its depth-camera coordinates mapped by the
 * depth-to-colour extrinsic, projected with the colour intrinsics, the image
 * sampled bilinearly from the 2x2 pixels at the floor of the position (inside
 * the image); each channel keeps the running mean (w c + c_obs) / (w + 1) in
 * fp32 rounded half up to 8 bits, the colour weight counting observations up
 * to max_w.  Constant observation weight (weight_mode 0) only; not with
 * swapping or batches.
 * ---------------------------------------------------------------------- */

/* Allocates the colour voxels (num_blocks x 512 x 4 bytes: r, g, b, colour
 * weight), all 0.  ITM_ERR_ARG when colour is already on, weight_mode is 1 or
 * swapping is on; ITM_ERR_CUDA when the memory cannot be had.  Freed with the
 * scene; itm_scene_reset clears it. */
int itm_colour_enable(itm_scene *scene);

/* itm_integrate plus the colour of an RGB frame: rgb_dev (device uint8
 * [intr_colour.height][intr_colour.width][3], row-major r, g, b) seen by a
 * camera with intrinsics intr_colour at T_d2c (host float[16], row-major
 * rigid map from depth-camera to colour-camera coordinates).  Asynchronous;
 * ITM_ERR_ARG when colour is off or an argument is invalid. */
int itm_integrate_colour(itm_scene *scene, const float *depth_dev, const itm_intrinsics *intr, const float T_wc[16],
                         const uint8_t *rgb_dev, const itm_intrinsics *intr_colour, const float T_d2c[16],
                         itm_stream stream);

/* Colour of the voxel nearest each of n world points (device float4[n]:
 * x, y, z, valid > 0 -- e.g. a raycast's vertex map), written as r, g, b,
 * colour weight to rgbw_dev (device uint8[n][4], 4-byte aligned); 0 where
 * the point is invalid or its block is not allocated.  Voxel coordinates as
 * in the raycast (p * (1/s)), nearest voxel floor(q + 1/2). */
int itm_colour_at(itm_scene *scene, const float *points_dev, int64_t n, uint8_t *rgbw_dev, itm_stream stream);

/* Colour of the allocated blocks, in the order of itm_scene_export: coords
 * (host int16[cap][3]) and rgbw (host uint8[cap][512][4]); *n receives the
 * number of blocks (cap 0 with null arrays asks for it).  Waits for the
 * scene's last stream. */
int itm_scene_export_colour(itm_scene *scene, int16_t *coords_host, uint8_t *rgbw_host, int cap, int *n);

/* ------------------------------------------------------------------------
 * Sec. 5 swapping: only the active part of the map stays in device memory;
 * the rest lives in a host block store with one slot per hash entry (the
 * paper's objective O2: a hash entry index is the host address).  A
 * swapped-out block keeps its hash entry with ptr -1 (Sec. 3.2).  Per frame:
 * itm_allocate (a segment that meets a swapped-out key gives its entry a
 * fresh device block and marks the host data as waiting), itm_swap_in,
 * itm_integrate, itm_raycast, itm_swap_out -- the order of the paper's
 * swapping pipeline.  itm_process_frame* do not swap; batches
 * (itm_batch_run) reject scenes with swapping on.
 *
 * The store is pinned host memory mapped into the device: the swap kernels
 * read and write a block's slot directly, so the host does no per-block work
 * and no transfer buffers are staged; each call moves at most
 * transfer_blocks blocks (objective O1).  Blocks are taken bucket by bucket
 * and, within a chain, in ascending key order (x, y, z as unsigned 16-bit
 * fields, z most significant), an order fixed by the set of keys.
 * ---------------------------------------------------------------------- */

/* Turns swapping on: allocates the host store ((num_buckets + num_excess) x
 * 512 x (4 + weight bytes), pinned and mapped) and the device state.
 * transfer_blocks (1 .. 2^24): blocks moved per call at most.  idle_frames
 * (>= 0): a block leaves the device once no allocation segment has met it
 * for that many allocations (0: every block without waiting host data is a
 * candidate).  ITM_ERR_ARG when swapping is already on or an argument is out
 * of range, ITM_ERR_CUDA when the memory cannot be had.  Freed with the
 * scene; itm_scene_reset clears it. */
int itm_swap_enable(itm_scene *scene, int transfer_blocks, int idle_frames);

/* The secondary integration of Sec. 5: up to transfer_blocks blocks whose
 * host data is waiting are fused into their device blocks, per voxel
 * F = (W_d F_d + W_h F_h) / (W_d + W_h), W = min(W_d + W_h, max_w), each
 * operation rounded on its own (a voxel the host never observed keeps the
 * device value; one the device has not observed takes the host value).
 * Asynchronous on stream; ITM_ERR_ARG when swapping is off. */
int itm_swap_in(itm_scene *scene, itm_stream stream);

/* Moves up to transfer_blocks blocks to their host slots: blocks in device
 * memory with no host data waiting that no allocation segment met in the
 * last idle_frames allocations.  Their entries keep their keys with ptr -1,
 * their device blocks are reset (sdf 1, weight 0) and return to the free
 * list.  Asynchronous on stream; ITM_ERR_ARG when swapping is off. */
int itm_swap_out(itm_scene *scene, itm_stream stream);

typedef struct {
    int64_t host_data;    /* entries with host data (swapped out or waiting) */
    int64_t swapped_out;  /* entries whose block is in the host store only */
    int64_t waiting;      /* entries with a device block and host data to fuse */
    int64_t moved_in;     /* blocks fused in since swapping was enabled */
    int64_t moved_out;    /* blocks moved to the host since swapping was enabled */
} itm_swap_counters;

/* Waits for the scene's last stream; ITM_ERR_ARG when swapping is off. */
int itm_swap_get_counters(itm_scene *scene, itm_swap_counters *out);

/* The host slots of the entries with host data, in entry order: coords
 * (host int16[cap][3]), sdf (host float[cap][512]), weights (host
 * uint8[cap][512] or float[cap][512] by weight_mode) and state (host
 * int32[cap]: 1 swapped out, 2 waiting).  *n receives the count;
 * ITM_ERR_TOO_LARGE when it exceeds cap (cap 0 with null arrays asks for the
 * count).  Waits for the scene's last stream. */
int itm_swap_export_host(itm_scene *scene, int16_t *coords_host, float *sdf_host, void *w_host,
                         int32_t *state_host, int cap, int *n);

#ifdef __cplusplus
}
#endif
#endif /* ITM_H */
