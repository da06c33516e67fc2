/*
 * itm_oracle.c -- plain, slow, single-threaded CPU oracle for the hashed-TSDF
 * per-frame core of InfiniTAM v3 (Prisacariu et al., 2017).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
 * bench's CPU-baseline leg may load this library.  It shares no code, header,
 * table or constant with the CUDA path; both sides receive the same seeded
 * inputs (depth frames, poses, parameters) and nothing else.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC
 * (no FMA contraction: every float operation below is rounded on its own, in
 * the order written, which is what makes the integer decisions reproducible).
 * The same source built with -fopenmp is the multi-threaded CPU baseline:
 * integration runs over blocks and the raycast over image rows in parallel
 * (each voxel and each pixel is computed alone, so nothing changes), and the
 * allocation records each row's blocks in parallel and inserts them afterwards
 * in the single-threaded order, so the hash table comes out byte-identical.
 *
 * What each function follows:
 *   orc_hash_index        Sec. 3.2, the printed hashIndex function
 *   lookup / insert       Sec. 3.3 (retrieval walks bucket then excess chain,
 *                         excess entry k >= 1 lives at num_buckets + k - 1,
 *                         a chain ends when offset < 1; insertion reserves
 *                         from prepopulated free lists)
 *   orc_allocate          Sec. 4.2 (segment d-mu .. d+mu per depth pixel,
 *                         every intersected block allocated)
 *   orc_integrate         Sec. 4.3 listing computeUpdatedVoxelDepthInfo
 *   orc_raycast           Sec. 4.4 state machine + two trilinear steps
 *   orc_raycast_combined  Sec. 7.2 combined TSDF of posed submaps, raycast
 *                         with the Sec. 4.4 state machine
 *   orc_icp_reduce/track  Sec. 4.1.1 depth tracker: point-to-plane sums over
 *                         the raycast maps, Gauss-Newton steps, pyramid
 *   orc_mesh              Sec. 4 Marching Cubes over the allocated blocks
 *   orc_depth_u16_to_f32  Sec. 4 (ViewBuilder: unsigned short -> float depth)
 *   orc_integrate_colour  Sec. 3.1 colour voxel (RGB + colour weight) fused
 *                         from an RGB frame beside the depth integration
 *   orc_swap_*            Sec. 5 swapping: a host block store with one slot
 *                         per hash entry, entries of swapped-out blocks kept
 *                         with ptr -1, at most K blocks moved per call, and
 *                         the secondary fusion of host data into a device
 *                         block that went on integrating meanwhile
 *
 * Readings taken where the paper is silent (each one is also listed in the
 * repository's design notes):
 *   - voxel g (global integer index) sits at world position (float)g * s
 *     (corner convention); block b holds voxels 8b .. 8b+7 per axis;
 *   - allocation: both ends of the segment are points on the pixel's ray at
 *     z-depth d-mu and d+mu; the blocks between them are enumerated with a
 *     3D DDA (Amanatides & Woo 1987) that only steps along axes which still
 *     have blocks left to cover; every block of the union over all pixels is
 *     allocated (the paper lets intra-frame colliding blocks wait for the next
 *     frame; here allocation is complete and deterministic);
 *   - integration visits every allocated block (the paper's visible list is
 *     an optimisation that must not change the result);
 *   - depth that is not > 0 (zero, negative or NaN) is no measurement;
 *   - learned weights: newW = w_px instead of 1, skipped when w_px <= 0;
 *   - raycast: see the comment above orc_raycast;
 *   - swapping: see the comment above orc_swap_enable;
 *   - colour: see the comment above orc_colour_enable.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_BLOCK 8
#define ORC_BLOCK3 512

enum {
    ORC_ST_HASH_FULL = 1,   /* excess list exhausted */
    ORC_ST_VBA_FULL = 2,    /* voxel block array exhausted */
    ORC_ST_RANGE = 4,       /* block coordinate outside int16 */
};

typedef struct {
    int16_t x, y, z, pad;
    int32_t offset; /* 0: no successor; k >= 1: next entry at nb + k - 1 */
    int32_t ptr;    /* >= 0 block index, -1 swapped out, < -1 unallocated */
} orc_entry;

typedef struct {
    float voxel_size, mu;
    int max_w;
    int nb, ne, nv;
    float z_min, z_max;
    orc_entry *entries;
    int32_t *excess_free; /* stack of free excess slots (0-based), top at excess_top-1 */
    int excess_top;
    int32_t *block_free;  /* stack of free block indices, top at block_top-1 */
    int block_top;
    float *sdf;           /* nv * 512, initialised when the block is handed out */
    float *w;
    int16_t *block_pos;   /* nv * 3: coordinates of the block owning each index */
    int32_t *alloc_order; /* block indices in order of allocation */
    int n_alloc;
    int status;
    /* Sec. 5 swapping, off until orc_swap_enable */
    int swap_on, swap_k, swap_idle;
    int frame;            /* allocations since swapping was enabled */
    uint8_t *swap_state;  /* per entry: ORC_SW_* */
    int32_t *touch;       /* per entry: last allocation whose segments met the block */
    float **host;         /* per entry: the host slot (512 sdf then 512 weights), made on first use */
    long long swapped_in, swapped_out;
    uint8_t *rgbw;        /* colour voxels (orc_colour_enable): nv * 512 * {r, g, b, colour weight} */
    /* one part of a scene split over shard_n processes by slabs of shard_w
     * blocks along x (orc_scene_set_shard); shard_n <= 1: the whole scene */
    int shard_n, shard_i, shard_w;
} orc_scene;

enum {
    ORC_SW_DEVICE = 0, /* the block's current data is in the device block (or it has none) */
    ORC_SW_HOST = 1,   /* swapped out: the data is in the host slot only (entry ptr -1) */
    ORC_SW_MERGE = 2,  /* host data waiting to be fused into the device block */
};

/* ---------------------------------------------------------------- hashing */

/* Sec. 3.2: xor of the coordinates times three primes, masked by nb-1. */
uint32_t orc_hash_index(int x, int y, int z, uint32_t mask)
{
    uint32_t hx = (uint32_t)x * 73856093u;
    uint32_t hy = (uint32_t)y * 19349669u;
    uint32_t hz = (uint32_t)z * 83492791u;
    return (hx ^ hy ^ hz) & mask;
}

orc_scene *orc_scene_new(float voxel_size, float mu, int max_w, int nb, int ne, int nv,
                         float z_min, float z_max)
{
    if (nb <= 0 || (nb & (nb - 1)) != 0 || ne < 0 || nv < 0) return NULL;
    orc_scene *s = (orc_scene *)calloc(1, sizeof(orc_scene));
    s->voxel_size = voxel_size;
    s->mu = mu;
    s->max_w = max_w;
    s->nb = nb;
    s->ne = ne;
    s->nv = nv;
    s->z_min = z_min;
    s->z_max = z_max;
    s->entries = (orc_entry *)malloc(sizeof(orc_entry) * (size_t)(nb + ne));
    for (int i = 0; i < nb + ne; ++i) {
        s->entries[i].x = s->entries[i].y = s->entries[i].z = s->entries[i].pad = 0;
        s->entries[i].offset = 0;
        s->entries[i].ptr = -2;
    }
    s->excess_free = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne > 0 ? ne : 1));
    for (int i = 0; i < ne; ++i) s->excess_free[i] = ne - 1 - i; /* pops 0,1,2,... */
    s->excess_top = ne;
    s->block_free = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    for (int i = 0; i < nv; ++i) s->block_free[i] = nv - 1 - i;
    s->block_top = nv;
    s->sdf = (float *)malloc(sizeof(float) * (size_t)(nv > 0 ? nv : 1) * ORC_BLOCK3);
    s->w = (float *)malloc(sizeof(float) * (size_t)(nv > 0 ? nv : 1) * ORC_BLOCK3);
    s->block_pos = (int16_t *)malloc(sizeof(int16_t) * 3 * (size_t)(nv > 0 ? nv : 1));
    s->alloc_order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    return s;
}

void orc_scene_free(orc_scene *s)
{
    if (!s) return;
    free(s->entries);
    free(s->excess_free);
    free(s->block_free);
    free(s->sdf);
    free(s->w);
    free(s->block_pos);
    free(s->alloc_order);
    if (s->host)
        for (int i = 0; i < s->nb + s->ne; ++i) free(s->host[i]);
    free(s->host);
    free(s->swap_state);
    free(s->touch);
    free(s->rgbw);
    free(s);
}

/* Sec. 3.3 retrieval: bucket, then the excess chain.  Returns the block index
 * (>= 0) or -1 when the block is not present. */
static int lookup(const orc_scene *s, int bx, int by, int bz)
{
    int idx = (int)orc_hash_index(bx, by, bz, (uint32_t)(s->nb - 1));
    for (;;) {
        const orc_entry *e = &s->entries[idx];
        if (e->x == bx && e->y == by && e->z == bz && e->ptr >= 0) return e->ptr;
        if (e->offset < 1) return -1;
        idx = s->nb + e->offset - 1;
    }
}

static int take_block(orc_scene *s, int bx, int by, int bz)
{
    if (s->block_top <= 0) {
        s->status |= ORC_ST_VBA_FULL;
        return -1;
    }
    int ptr = s->block_free[--s->block_top];
    for (int i = 0; i < ORC_BLOCK3; ++i) {
        s->sdf[(size_t)ptr * ORC_BLOCK3 + i] = 1.0f; /* Sec. 3.1: float sdf starts at 1 */
        s->w[(size_t)ptr * ORC_BLOCK3 + i] = 0.0f;
    }
    if (s->rgbw) memset(&s->rgbw[(size_t)ptr * ORC_BLOCK3 * 4], 0, ORC_BLOCK3 * 4); /* no colour observed */
    s->block_pos[3 * ptr + 0] = (int16_t)bx;
    s->block_pos[3 * ptr + 1] = (int16_t)by;
    s->block_pos[3 * ptr + 2] = (int16_t)bz;
    s->alloc_order[s->n_alloc++] = ptr;
    return ptr;
}

static void touch_entry(orc_scene *s, const orc_entry *e)
{
    if (s->swap_on) s->touch[e - s->entries] = s->frame;
}

/* Sec. 3.3 insertion: claim the bucket if it is free, otherwise walk to the
 * chain's end, reserve an excess entry and link it from the last entry.  With
 * swapping (Sec. 5), a key whose entry is swapped out (ptr -1) keeps that
 * entry: it gets a fresh device block and waits for its host data to be
 * fused in (ORC_SW_MERGE).  Every block met is stamped with the frame. */
static void insert_if_missing(orc_scene *s, int bx, int by, int bz)
{
    int idx = (int)orc_hash_index(bx, by, bz, (uint32_t)(s->nb - 1));
    orc_entry *e = &s->entries[idx];
    if (e->ptr < -1) { /* the bucket itself is unused */
        if (s->block_top <= 0) {
            s->status |= ORC_ST_VBA_FULL;
            return;
        }
        e->x = (int16_t)bx;
        e->y = (int16_t)by;
        e->z = (int16_t)bz;
        e->ptr = take_block(s, bx, by, bz);
        touch_entry(s, e);
        return;
    }
    for (;;) {
        if (e->x == bx && e->y == by && e->z == bz) { /* present */
            if (e->ptr == -1) {
                if (s->block_top <= 0) {
                    s->status |= ORC_ST_VBA_FULL;
                    return;
                }
                e->ptr = take_block(s, bx, by, bz);
                s->swap_state[e - s->entries] = ORC_SW_MERGE;
            }
            touch_entry(s, e);
            return;
        }
        if (e->offset < 1) break;
        e = &s->entries[s->nb + e->offset - 1];
    }
    if (s->excess_top <= 0) {
        s->status |= ORC_ST_HASH_FULL;
        return;
    }
    if (s->block_top <= 0) {
        s->status |= ORC_ST_VBA_FULL;
        return;
    }
    int slot = s->excess_free[--s->excess_top];
    orc_entry *n = &s->entries[s->nb + slot];
    n->x = (int16_t)bx;
    n->y = (int16_t)by;
    n->z = (int16_t)bz;
    n->offset = 0;
    n->ptr = take_block(s, bx, by, bz);
    e->offset = slot + 1;
    touch_entry(s, n);
}

/* ------------------------------------------------------------ pose helpers */

/* M = T^-1 for a rigid camera-to-world T, computed in fp64 as [R^T, -R^T t]
 * and rounded once to float. */
static void rigid_inverse(const float T[16], float M[16])
{
    double R[3][3], t[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) R[i][j] = (double)T[4 * i + j];
        t[i] = (double)T[4 * i + 3];
    }
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) M[4 * i + j] = (float)R[j][i];
        double acc = 0.0;
        for (int j = 0; j < 3; ++j) acc -= R[j][i] * t[j];
        M[4 * i + 3] = (float)acc;
    }
    M[12] = M[13] = M[14] = 0.0f;
    M[15] = 1.0f;
}

/* Row i of a 4x4 float matrix applied to (x, y, z, 1): ((a*x + b*y) + c*z) + d,
 * each operation rounded separately. */
static float row_apply(const float *m, float x, float y, float z)
{
    float a = m[0] * x;
    float b = m[1] * y;
    float c = m[2] * z;
    float r = a + b;
    r = r + c;
    r = r + m[3];
    return r;
}

static int in_i16(int v) { return v >= -32768 && v <= 32767; }

/* -------------------------------------------------------------- allocation */

/* Where the blocks a segment crosses go: NULL inserts each into the scene at
 * once; a list records them (with the status bits they raised) so that they
 * can be inserted later in the same order. */
typedef struct {
    int16_t *xyz;
    int n, cap;
    int status;
} block_list;

/* ------------------------------------------------------ slab partition
 *
 * A scene split over n parts (not in the paper; the multi-process form of
 * the per-frame core): block column x belongs to part floor(x / w) mod n.
 * Part i keeps the blocks of its own columns and of the ORC_SHARD_GHOST
 * columns on either side, so that every trilinear sample, refinement step and
 * normal of a point in its own columns reads the same voxels as the whole
 * scene (each kept block's voxels equal the whole scene's bit for bit); its
 * raycast reports only hits whose block is its own, and the parts' maps are
 * merged per pixel by the hit nearest to the camera.  The merged map is close
 * to the whole scene's but not the same computation: a ray that reaches a
 * part's columns from space the part does not hold starts its fine search
 * there, so near the slab boundaries its refined hit can differ by a few mm
 * (and rarely hit or miss differently). */
static int slab_owner(int bx, int n, int w)
{
    int q = bx >= 0 ? bx / w : -((-bx + w - 1) / w); /* floor(bx / w) */
    int r = q % n;
    return r < 0 ? r + n : r;
}

#define ORC_SHARD_GHOST 1

static int shard_keeps(const orc_scene *s, int bx)
{
    if (s->shard_n <= 1) return 1;
    for (int d = -ORC_SHARD_GHOST; d <= ORC_SHARD_GHOST; ++d)
        if (slab_owner(bx + d, s->shard_n, s->shard_w) == s->shard_i) return 1;
    return 0;
}

static int shard_owns(const orc_scene *s, int bx)
{
    return s->shard_n <= 1 || slab_owner(bx, s->shard_n, s->shard_w) == s->shard_i;
}

int orc_scene_set_shard(orc_scene *s, int n, int i, int w)
{
    if (n < 1 || i < 0 || i >= n || w < 2) return -1;
    s->shard_n = n;
    s->shard_i = i;
    s->shard_w = w;
    return 0;
}

static void emit_block(orc_scene *s, block_list *out, int bx, int by, int bz)
{
    if (!shard_keeps(s, bx)) return;
    if (!out) {
        insert_if_missing(s, bx, by, bz);
        return;
    }
    if (out->n == out->cap) {
        int cap = out->cap ? 2 * out->cap : 1024;
        int16_t *p = (int16_t *)realloc(out->xyz, (size_t)cap * 3 * sizeof(int16_t));
        if (!p) abort();
        out->xyz = p;
        out->cap = cap;
    }
    out->xyz[3 * out->n + 0] = (int16_t)bx;
    out->xyz[3 * out->n + 1] = (int16_t)by;
    out->xyz[3 * out->n + 2] = (int16_t)bz;
    out->n += 1;
}

/* Blocks crossed by the segment q0 -> q1 (block units), stepping one axis at a
 * time towards the end block; ties go to x, then y, then z. */
static void dda_blocks(orc_scene *s, block_list *out, const float q0[3], const float q1[3])
{
    int cur[3], end[3], step[3], left[3];
    float tmax[3], tdelta[3];
    for (int i = 0; i < 3; ++i) {
        float f0 = floorf(q0[i]);
        float f1 = floorf(q1[i]);
        if (!(f0 >= -32768.0f && f0 <= 32767.0f && f1 >= -32768.0f && f1 <= 32767.0f)) {
            if (out) out->status |= ORC_ST_RANGE;
            else s->status |= ORC_ST_RANGE;
            return;
        }
        cur[i] = (int)f0;
        end[i] = (int)f1;
        float dir = q1[i] - q0[i];
        if (end[i] > cur[i]) {
            step[i] = 1;
            left[i] = end[i] - cur[i];
            tdelta[i] = 1.0f / dir;
            tmax[i] = ((float)(cur[i] + 1) - q0[i]) / dir;
        } else if (end[i] < cur[i]) {
            step[i] = -1;
            left[i] = cur[i] - end[i];
            tdelta[i] = -1.0f / dir;
            tmax[i] = ((float)cur[i] - q0[i]) / dir;
        } else {
            step[i] = 0;
            left[i] = 0;
            tdelta[i] = 0.0f;
            tmax[i] = 0.0f;
        }
    }
    emit_block(s, out, cur[0], cur[1], cur[2]);
    while (left[0] + left[1] + left[2] > 0) {
        int a = -1;
        for (int i = 0; i < 3; ++i)
            if (left[i] > 0 && (a < 0 || tmax[i] < tmax[a])) a = i;
        cur[a] += step[a];
        tmax[a] = tmax[a] + tdelta[a];
        left[a] -= 1;
        emit_block(s, out, cur[0], cur[1], cur[2]);
    }
}

/* Sec. 4.2, first part, for pixel (u, v): the ends of the line from depth
 * d-mu to d+mu on the pixel's ray, in block units.  Returns 0 when the pixel
 * has no measurement in [z_min, z_max]. */
static int pixel_segment(const orc_scene *s, const float *depth, int W, int u, int v, const float intr[4],
                         const float T_wc[16], float inv_b, float q0[3], float q1[3])
{
    const float fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3];
    const float mu = s->mu;
    float d = depth[(size_t)v * W + u];
    if (!(d > 0.0f)) return 0;
    if (d < s->z_min || d > s->z_max) return 0;
    float rx = ((float)u - cx) / fx;
    float ry = ((float)v - cy) / fy;
    float z0 = d - mu;
    float z1 = d + mu;
    if (z0 < 1e-3f) z0 = 1e-3f;
    for (int i = 0; i < 3; ++i) {
        float p0 = row_apply(&T_wc[4 * i], rx * z0, ry * z0, z0);
        float p1 = row_apply(&T_wc[4 * i], rx * z1, ry * z1, z1);
        q0[i] = p0 * inv_b;
        q1[i] = p1 * inv_b;
    }
    return 1;
}

/* Sec. 4.2, first and second parts: for each valid pixel, the line from
 * depth d-mu to d+mu on the pixel's ray; every block it crosses is looked up
 * and inserted when missing.  Pixels are visited in row-major order.
 * Returns the sticky status bits. */
int orc_allocate(orc_scene *s, const float *depth, int W, int H, const float intr[4],
                 const float T_wc[16])
{
    const float inv_b = (float)(1.0 / (8.0 * (double)s->voxel_size));
    if (s->swap_on) ++s->frame;
#ifndef _OPENMP
    for (int v = 0; v < H; ++v) {
        for (int u = 0; u < W; ++u) {
            float q0[3], q1[3];
            if (pixel_segment(s, depth, W, u, v, intr, T_wc, inv_b, q0, q1)) dda_blocks(s, NULL, q0, q1);
        }
    }
#else
    /* the crossed blocks of each row, found in parallel, then inserted in
     * row-major order: the insertions and their order are those above */
    block_list *rows = (block_list *)calloc((size_t)(H > 0 ? H : 1), sizeof(block_list));
    if (!rows) abort();
#pragma omp parallel for schedule(dynamic, 4)
    for (int v = 0; v < H; ++v) {
        for (int u = 0; u < W; ++u) {
            float q0[3], q1[3];
            if (pixel_segment(s, depth, W, u, v, intr, T_wc, inv_b, q0, q1)) dda_blocks(s, &rows[v], q0, q1);
        }
    }
    for (int v = 0; v < H; ++v) {
        for (int i = 0; i < rows[v].n; ++i)
            insert_if_missing(s, rows[v].xyz[3 * i], rows[v].xyz[3 * i + 1], rows[v].xyz[3 * i + 2]);
        s->status |= rows[v].status;
        free(rows[v].xyz);
    }
    free(rows);
#endif
    return s->status;
}

/* Threads the parallel loops use: 1 in the plain build. */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------- integration */

static int coord_ok(float q);

/* An RGB frame for the colour integration: 8-bit r, g, b per pixel
 * (row-major, Wc x Hc), its intrinsics and the rigid map from depth-camera to
 * colour-camera coordinates. */
typedef struct {
    const uint8_t *rgb;
    int Wc, Hc;
    float fx, fy, cx, cy;
    float T[16];
} colour_frame;

/* Colour of voxel i of block ptr from the colour frame, the voxel at
 * depth-camera coordinates (X, Y, Z).  Readings: the point maps into the
 * colour camera by T (rows applied as row_apply), projects with the colour
 * intrinsics and samples the image bilinearly (the 2x2 pixels at floor(u),
 * floor(v) must be inside the image); each channel takes the running mean
 * (w c + c_obs) / (w + 1) rounded half up to 8 bits, and the colour weight
 * w grows by one up to max_w. */
static void colour_update(orc_scene *s, int ptr, int i, float X, float Y, float Z, const colour_frame *cf)
{
    float Xc = row_apply(&cf->T[0], X, Y, Z);
    float Yc = row_apply(&cf->T[4], X, Y, Z);
    float Zc = row_apply(&cf->T[8], X, Y, Z);
    if (!(Zc > 0.0f)) return;
    float uc = (cf->fx * Xc) / Zc + cf->cx;
    float vc = (cf->fy * Yc) / Zc + cf->cy;
    if (!(uc >= 0.0f && vc >= 0.0f && uc < (float)(cf->Wc - 1) && vc < (float)(cf->Hc - 1))) return;
    int u0 = (int)uc, v0 = (int)vc;
    float a = uc - (float)u0, b = vc - (float)v0;
    uint8_t *c = &s->rgbw[((size_t)ptr * ORC_BLOCK3 + i) * 4];
    float wc = (float)c[3];
    for (int ch = 0; ch < 3; ++ch) {
        const uint8_t *P = cf->rgb;
        float p00 = (float)P[((size_t)v0 * cf->Wc + u0) * 3 + ch];
        float p10 = (float)P[((size_t)v0 * cf->Wc + u0 + 1) * 3 + ch];
        float p01 = (float)P[((size_t)(v0 + 1) * cf->Wc + u0) * 3 + ch];
        float p11 = (float)P[((size_t)(v0 + 1) * cf->Wc + u0 + 1) * 3 + ch];
        float top = p00 + a * (p10 - p00);
        float bot = p01 + a * (p11 - p01);
        float obs = top + b * (bot - top);
        float nc = (wc * (float)c[ch] + obs) / (wc + 1.0f);
        int q = (int)(nc + 0.5f);
        c[ch] = (uint8_t)(q < 0 ? 0 : (q > 255 ? 255 : q));
    }
    float nw = wc + 1.0f;
    c[3] = (uint8_t)(nw < (float)s->max_w ? nw : (float)s->max_w);
}

/* Sec. 4.3: computeUpdatedVoxelDepthInfo applied to every voxel of every
 * allocated block.  wpx (nullable) holds a per-pixel observation weight that
 * replaces the constant 1 (learned-confidence mode); cf (nullable) an RGB
 * frame whose colour is fused into the voxels that get a depth update within
 * the band |eta| <= mu.  Returns the number of voxels updated. */
static long long integrate_impl(orc_scene *s, const float *depth, int W, int H, const float intr[4],
                                const float T_wc[16], const float *wpx, const colour_frame *cf)
{
    float M[16];
    rigid_inverse(T_wc, M);
    const float fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3];
    const float mu = s->mu;
    const float vs = s->voxel_size;
    const float max_w = (float)s->max_w;
    const float umax = (float)(W - 2), vmax = (float)(H - 2);
    long long updated = 0;
#pragma omp parallel for reduction(+ : updated) schedule(dynamic, 16)
    for (int k = 0; k < s->n_alloc; ++k) {
        int ptr = s->alloc_order[k];
        int bx = s->block_pos[3 * ptr], by = s->block_pos[3 * ptr + 1], bz = s->block_pos[3 * ptr + 2];
        float *F = &s->sdf[(size_t)ptr * ORC_BLOCK3];
        float *Wt = &s->w[(size_t)ptr * ORC_BLOCK3];
        for (int lz = 0; lz < 8; ++lz)
            for (int ly = 0; ly < 8; ++ly)
                for (int lx = 0; lx < 8; ++lx) {
                    int i = lx + 8 * ly + 64 * lz;
                    float px = (float)(bx * 8 + lx) * vs;
                    float py = (float)(by * 8 + ly) * vs;
                    float pz = (float)(bz * 8 + lz) * vs;
                    float X = row_apply(&M[0], px, py, pz);
                    float Y = row_apply(&M[4], px, py, pz);
                    float Z = row_apply(&M[8], px, py, pz);
                    if (Z <= 0.0f) continue;
                    float u = (fx * X) / Z + cx;
                    float v = (fy * Y) / Z + cy;
                    if (u < 1.0f || u > umax || v < 1.0f || v > vmax) continue;
                    int pix = (int)(u + 0.5f) + (int)(v + 0.5f) * W;
                    float d = depth[pix];
                    if (!(d > 0.0f)) continue;
                    float eta = d - Z;
                    if (eta < -mu) continue;
                    float obs = 1.0f;
                    if (wpx) {
                        obs = wpx[pix];
                        if (!(obs > 0.0f)) continue;
                    }
                    float f = eta / mu;
                    if (f > 1.0f) f = 1.0f;
                    float oldW = Wt[i];
                    float num = oldW * F[i] + obs * f;
                    float den = oldW + obs;
                    F[i] = num / den;
                    Wt[i] = den < max_w ? den : max_w;
                    ++updated;
                    if (cf && eta <= mu) colour_update(s, ptr, i, X, Y, Z, cf);
                }
    }
    return updated;
}

long long orc_integrate(orc_scene *s, const float *depth, int W, int H, const float intr[4],
                        const float T_wc[16], const float *wpx)
{
    return integrate_impl(s, depth, W, H, intr, T_wc, wpx, NULL);
}

/* Colour voxels (Sec. 3.1: the voxel types with colour carry an RGB value and
 * a colour weight).  The paper gives the voxel, not its update; the readings
 * are at colour_update.  Blocks start with colour 0 and colour weight 0. */
int orc_colour_enable(orc_scene *s)
{
    if (s->rgbw) return -1;
    s->rgbw = (uint8_t *)calloc((size_t)(s->nv > 0 ? s->nv : 1) * ORC_BLOCK3 * 4, 1);
    return 0;
}

/* The depth integration of orc_integrate plus the colour of an RGB frame
 * (rgb: Hc x Wc x 3 bytes; intr_c: fx, fy, cx, cy; T_d2c: depth-camera to
 * colour-camera rigid map, row-major). */
long long orc_integrate_colour(orc_scene *s, const float *depth, int W, int H, const float intr[4],
                               const float T_wc[16], const uint8_t *rgb, int Wc, int Hc, const float intr_c[4],
                               const float T_d2c[16])
{
    if (!s->rgbw) return -1;
    colour_frame cf;
    cf.rgb = rgb;
    cf.Wc = Wc;
    cf.Hc = Hc;
    cf.fx = intr_c[0];
    cf.fy = intr_c[1];
    cf.cx = intr_c[2];
    cf.cy = intr_c[3];
    memcpy(cf.T, T_d2c, sizeof(cf.T));
    return integrate_impl(s, depth, W, H, intr, T_wc, NULL, &cf);
}

/* Colour at n world points (x, y, z, valid; e.g. a raycast's vertex map):
 * the colour voxel nearest to each valid point, r, g, b, colour weight; 0
 * where the point is invalid or its voxel's block is not allocated.  Voxel
 * coordinates q = p * (1/s) as in the raycast, nearest voxel floor(q + 1/2). */
void orc_colour_at(const orc_scene *s, const float *pts, long long n, uint8_t *out)
{
    const float inv_s = (float)(1.0 / (double)s->voxel_size);
    for (long long j = 0; j < n; ++j) {
        uint8_t *o = &out[4 * j];
        o[0] = o[1] = o[2] = o[3] = 0;
        if (!s->rgbw || !(pts[4 * j + 3] > 0.0f)) continue;
        int g[3];
        int ok = 1;
        for (int a = 0; a < 3; ++a) {
            float q = pts[4 * j + a] * inv_s;
            if (!coord_ok(q)) ok = 0;
            else g[a] = (int)floorf(q + 0.5f);
        }
        if (!ok) continue;
        int ptr = lookup(s, g[0] >> 3, g[1] >> 3, g[2] >> 3);
        if (ptr < 0) continue;
        memcpy(o, &s->rgbw[((size_t)ptr * ORC_BLOCK3 + (g[0] & 7) + 8 * (g[1] & 7) + 64 * (g[2] & 7)) * 4], 4);
    }
}

/* ----------------------------------------------------------------- raycast */

/* The TSDF as a field: the stored value of voxel g when its block is
 * allocated, otherwise the default voxel's value 1 (Sec. 3.3: retrieval of a
 * missing block returns a default-constructed voxel). */
static float voxel_value(const orc_scene *s, int gx, int gy, int gz, int *observed)
{
    int ptr = lookup(s, gx >> 3, gy >> 3, gz >> 3);
    if (ptr < 0) {
        *observed = 0;
        return 1.0f;
    }
    size_t i = (size_t)ptr * ORC_BLOCK3 + (gx & 7) + 8 * (gy & 7) + 64 * (gz & 7);
    *observed = s->w[i] > 0.0f;
    return s->sdf[i];
}

static int coord_ok(float q) { return q > -262000.0f && q < 262000.0f; }

static float lerpf(float a, float b, float t) { return a + t * (b - a); }

/* Trilinear interpolation of the field at voxel coordinates q.  *all_obs is
 * cleared when one of the eight voxels is unallocated or was never observed. */
static float trilinear(const orc_scene *s, const float q[3], int *all_obs)
{
    float g0f[3], fr[3];
    for (int i = 0; i < 3; ++i) {
        g0f[i] = floorf(q[i]);
        fr[i] = q[i] - g0f[i];
    }
    int x = (int)g0f[0], y = (int)g0f[1], z = (int)g0f[2];
    int o[8];
    float c000 = voxel_value(s, x, y, z, &o[0]), c100 = voxel_value(s, x + 1, y, z, &o[1]);
    float c010 = voxel_value(s, x, y + 1, z, &o[2]), c110 = voxel_value(s, x + 1, y + 1, z, &o[3]);
    float c001 = voxel_value(s, x, y, z + 1, &o[4]), c101 = voxel_value(s, x + 1, y, z + 1, &o[5]);
    float c011 = voxel_value(s, x, y + 1, z + 1, &o[6]), c111 = voxel_value(s, x + 1, y + 1, z + 1, &o[7]);
    for (int i = 0; i < 8; ++i) *all_obs &= o[i];
    float c00 = lerpf(c000, c100, fr[0]);
    float c10 = lerpf(c010, c110, fr[0]);
    float c01 = lerpf(c001, c101, fr[0]);
    float c11 = lerpf(c011, c111, fr[0]);
    float c0 = lerpf(c00, c10, fr[1]);
    float c1 = lerpf(c01, c11, fr[1]);
    return lerpf(c0, c1, fr[2]);
}

enum { SEARCH_BLOCK_COARSE = 0, SEARCH_BLOCK_FINE, SEARCH_SURFACE, BEHIND_SURFACE, WRONG_SIDE };

/*
 * Sec. 4.4 raycast.  Readings (the paper names the states and the step
 * policy but not the constants):
 *   ray of pixel (u, v): o + t * dir, dir = R ((u-cx)/fx, (v-cy)/fy, 1), so t
 *   is z-depth; len = |((u-cx)/fx, (v-cy)/fy, 1)|; metric steps are divided by
 *   len once per ray: tB = 8s/len, tmu = mu/len, ts = s/len.
 *   t starts at z_min; the ray misses once t > z_max.
 *   Voxel coordinates q = p * (1/s); "the block at p" is the block of the
 *   nearest voxel floor(q + 0.5).
 *   COARSE : block unallocated -> t += tB; allocated -> t -= tB, go FINE.
 *   FINE   : block unallocated -> t += tmu; allocated -> read F (trilinear):
 *            F <= 0 -> WRONG_SIDE (no hit); else go SURFACE at the same t.
 *   SURFACE: block unallocated -> go COARSE (t unchanged); else read F
 *            (trilinear): F <= 0 -> BEHIND_SURFACE; else t += max(F*tmu, ts).
 *   BEHIND : twice t += F(t) * tmu with trilinear F; hit point o + t * dir.
 *   Normal : central differences of the trilinear field at +-1 voxel along
 *            each world axis, normalised.  No normal when the gradient is
 *            zero or when one of the 48 voxels read is unallocated or has
 *            weight 0 (its value is the default 1, not a measurement).
 *   At most 4*(z_max-z_min)/s + 64 iterations, then the ray misses.
 * Output: float4 per pixel, vertex (x, y, z, 1) / (0,0,0,0) on a miss and
 * normal (nx, ny, nz, 1) / (0,0,0,0) when absent.  Returns the hit count.
 */
int orc_raycast(const orc_scene *s, int W, int H, const float intr[4], const float T_wc[16],
                float *vtx, float *nrm)
{
    const float fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3];
    const float vs = s->voxel_size;
    const float inv_s = (float)(1.0 / (double)vs);
    const float B = 8.0f * vs;
    const float mu = s->mu;
    const int max_iter = (int)(4.0f * (s->z_max - s->z_min) / vs) + 64;
    int hits = 0;
#pragma omp parallel for reduction(+ : hits) schedule(dynamic, 2)
    for (int v = 0; v < H; ++v) {
        for (int u = 0; u < W; ++u) {
            size_t o4 = 4 * ((size_t)v * W + u);
            vtx[o4] = vtx[o4 + 1] = vtx[o4 + 2] = vtx[o4 + 3] = 0.0f;
            nrm[o4] = nrm[o4 + 1] = nrm[o4 + 2] = nrm[o4 + 3] = 0.0f;
            float dc0 = ((float)u - cx) / fx;
            float dc1 = ((float)v - cy) / fy;
            float len = sqrtf((dc0 * dc0 + dc1 * dc1) + 1.0f);
            float dir[3], org[3];
            for (int i = 0; i < 3; ++i) {
                dir[i] = (T_wc[4 * i] * dc0 + T_wc[4 * i + 1] * dc1) + T_wc[4 * i + 2];
                org[i] = T_wc[4 * i + 3];
            }
            const float tB = B / len, tmu = mu / len, ts = vs / len;
            float t = s->z_min;
            int state = SEARCH_BLOCK_COARSE;
            float q[3];
            int it = 0;
            for (; it < max_iter && t <= s->z_max; ++it) {
                int ok = 1;
                for (int i = 0; i < 3; ++i) {
                    q[i] = (org[i] + t * dir[i]) * inv_s;
                    ok &= coord_ok(q[i]);
                }
                int alloc = 0;
                if (ok) {
                    int nx = (int)floorf(q[0] + 0.5f), ny = (int)floorf(q[1] + 0.5f), nz = (int)floorf(q[2] + 0.5f);
                    int bx = nx >> 3, by = ny >> 3, bz = nz >> 3;
                    alloc = in_i16(bx) && in_i16(by) && in_i16(bz) && lookup(s, bx, by, bz) >= 0;
                }
                if (state == SEARCH_BLOCK_COARSE) {
                    if (!alloc) {
                        t = t + tB;
                    } else {
                        t = t - tB;
                        state = SEARCH_BLOCK_FINE;
                    }
                    continue;
                }
                if (!alloc) {
                    if (state == SEARCH_BLOCK_FINE) t = t + tmu;
                    else state = SEARCH_BLOCK_COARSE;
                    continue;
                }
                int obs = 1;
                float F = trilinear(s, q, &obs);
                if (state == SEARCH_BLOCK_FINE) {
                    if (F <= 0.0f) {
                        state = WRONG_SIDE;
                        break;
                    }
                    state = SEARCH_SURFACE;
                }
                if (F <= 0.0f) {
                    state = BEHIND_SURFACE;
                    break;
                }
                float step = F * tmu;
                if (step < ts) step = ts;
                t = t + step;
            }
            if (state != BEHIND_SURFACE) continue;
            for (int r = 0; r < 2; ++r) {
                for (int i = 0; i < 3; ++i) q[i] = (org[i] + t * dir[i]) * inv_s;
                int obs = 1;
                float F = trilinear(s, q, &obs);
                t = t + F * tmu;
            }
            float p[3];
            for (int i = 0; i < 3; ++i) {
                p[i] = org[i] + t * dir[i];
                q[i] = p[i] * inv_s;
            }
            if (!(coord_ok(q[0]) && coord_ok(q[1]) && coord_ok(q[2]))) continue;
            if (!shard_owns(s, ((int)floorf(q[0] + 0.5f)) >> 3)) continue; /* another part's hit */
            vtx[o4] = p[0];
            vtx[o4 + 1] = p[1];
            vtx[o4 + 2] = p[2];
            vtx[o4 + 3] = 1.0f;
            ++hits;
            float g[3];
            int obs = 1;
            for (int a = 0; a < 3; ++a) {
                float qp[3] = {q[0], q[1], q[2]}, qm[3] = {q[0], q[1], q[2]};
                qp[a] = q[a] + 1.0f;
                qm[a] = q[a] - 1.0f;
                float fp = trilinear(s, qp, &obs);
                float fm = trilinear(s, qm, &obs);
                g[a] = fp - fm;
            }
            float gl = sqrtf((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]);
            if (obs && gl > 0.0f) {
                nrm[o4] = g[0] / gl;
                nrm[o4 + 1] = g[1] / gl;
                nrm[o4 + 2] = g[2] / gl;
                nrm[o4 + 3] = 1.0f;
            }
        }
    }
    return hits;
}

/* The parts' raycasts (n maps of W x H float4 vertices and normals, one part
 * after another) merged: per pixel the hit nearest to the camera, its camera
 * depth z = row 2 of float(T_wc^-1) applied to the vertex; equal depths go to
 * the lower part.  No hit in any part: zeros. */
void orc_merge_raycasts(int n, const float *vtx, const float *nrm, int W, int H, const float T_wc[16],
                        float *vtx_out, float *nrm_out)
{
    float M[16];
    rigid_inverse(T_wc, M);
    const size_t np = (size_t)W * H;
    for (size_t o = 0; o < np; ++o) {
        int best = -1;
        float best_z = 0.0f;
        for (int k = 0; k < n; ++k) {
            const float *V = vtx + 4 * ((size_t)k * np + o);
            if (!(V[3] > 0.0f)) continue;
            const float z = row_apply(&M[8], V[0], V[1], V[2]);
            if (best < 0 || z < best_z) {
                best = k;
                best_z = z;
            }
        }
        for (int c = 0; c < 4; ++c) {
            vtx_out[4 * o + c] = best < 0 ? 0.0f : vtx[4 * ((size_t)best * np + o) + c];
            nrm_out[4 * o + c] = best < 0 ? 0.0f : nrm[4 * ((size_t)best * np + o) + c];
        }
    }
}

/* ------------------------------------------------------------ combined map */

/* Trilinear interpolation of the sdf and of the weight of one submap at its
 * voxel coordinates q, both over the same eight voxels and in the order of
 * trilinear(): an unallocated voxel has sdf 1 and weight 0. */
static void trilinear_fw(const orc_scene *s, const float q[3], float *F, float *Wt)
{
    float g0f[3], fr[3];
    for (int i = 0; i < 3; ++i) {
        g0f[i] = floorf(q[i]);
        fr[i] = q[i] - g0f[i];
    }
    int x = (int)g0f[0], y = (int)g0f[1], z = (int)g0f[2];
    float c[8], w[8];
    for (int k = 0; k < 8; ++k) {
        int gx = x + (k & 1), gy = y + ((k >> 1) & 1), gz = z + ((k >> 2) & 1);
        int ptr = lookup(s, gx >> 3, gy >> 3, gz >> 3);
        if (ptr < 0) {
            c[k] = 1.0f;
            w[k] = 0.0f;
        } else {
            size_t i = (size_t)ptr * ORC_BLOCK3 + (gx & 7) + 8 * (gy & 7) + 64 * (gz & 7);
            c[k] = s->sdf[i];
            w[k] = s->w[i];
        }
    }
    float v[2][8];
    for (int k = 0; k < 8; ++k) {
        v[0][k] = c[k];
        v[1][k] = w[k];
    }
    float out[2];
    for (int m = 0; m < 2; ++m) {
        float c00 = lerpf(v[m][0], v[m][1], fr[0]);
        float c10 = lerpf(v[m][2], v[m][3], fr[0]);
        float c01 = lerpf(v[m][4], v[m][5], fr[0]);
        float c11 = lerpf(v[m][6], v[m][7], fr[0]);
        float c0 = lerpf(c00, c10, fr[1]);
        float c1 = lerpf(c01, c11, fr[1]);
        out[m] = lerpf(c0, c1, fr[2]);
    }
    *F = out[0];
    *Wt = out[1];
}

/* Voxel coordinates of world point X in submap i: q = (P_i X) / s, with P_i
 * (row-major 4x4, submap-from-world) applied row by row as in row_apply.
 * Returns 0 when a coordinate is out of the representable range. */
static int submap_coords(const float *P, const float X[3], float inv_s, float q[3])
{
    int ok = 1;
    for (int r = 0; r < 3; ++r) {
        q[r] = row_apply(P + 4 * r, X[0], X[1], X[2]) * inv_s;
        ok &= coord_ok(q[r]);
    }
    return ok;
}

/* Is the block of the voxel nearest to X allocated in any submap? */
static int combined_alloc(const orc_scene *const *S, const float *P, int n, const float X[3], float inv_s)
{
    for (int i = 0; i < n; ++i) {
        float q[3];
        if (!submap_coords(P + 16 * i, X, inv_s, q)) continue;
        int bx = ((int)floorf(q[0] + 0.5f)) >> 3, by = ((int)floorf(q[1] + 0.5f)) >> 3,
            bz = ((int)floorf(q[2] + 0.5f)) >> 3;
        if (in_i16(bx) && in_i16(by) && in_i16(bz) && lookup(S[i], bx, by, bz) >= 0) return 1;
    }
    return 0;
}

/* Sec. 7.2 combined TSDF at world point X: sum over the submaps (in index
 * order) of W_i(P_i X) F_i(P_i X), divided by the sum of W_i(P_i X) so that
 * the value is a TSDF in [-1, 1] and the raycast's step rule keeps its
 * meaning (the printed sum is not normalised; dividing by a positive number
 * keeps its zero set).  With no weight anywhere (den = 0) the value is the
 * unobserved default 1.  *den receives the weight sum. */
float orc_combined_value(const orc_scene *const *S, const float *P, int n, const float X[3], float *den)
{
    const float inv_s = (float)(1.0 / (double)S[0]->voxel_size);
    float num = 0.0f, dsum = 0.0f;
    for (int i = 0; i < n; ++i) {
        float q[3];
        if (!submap_coords(P + 16 * i, X, inv_s, q)) continue;
        float F, Wt;
        trilinear_fw(S[i], q, &F, &Wt);
        num = num + Wt * F;
        dsum = dsum + Wt;
    }
    if (den) *den = dsum;
    return dsum > 0.0f ? num / dsum : 1.0f;
}

/*
 * Raycast of the combined map of n submaps (Sec. 7.2: the combined TSDF is
 * never built; it is a view over the submaps during rendering).  P holds n
 * row-major 4x4 submap-from-world poses; all submaps share voxel size, mu and
 * the depth range (those of S[0]).  The ray, step sizes, iteration limit,
 * states and refinement are those of orc_raycast, in world coordinates, with
 *   allocated(X) = the nearest voxel's block is allocated in some submap,
 *   F(X)         = orc_combined_value(X).
 * Normal: central differences of the combined value at X +- s along each
 * world axis, normalised; none when the gradient is zero or one of the six
 * samples has no weight in any submap.  Returns the hit count.
 */
int orc_raycast_combined(const orc_scene *const *S, const float *P, int n, int W, int H, const float intr[4],
                         const float T_wc[16], float *vtx, float *nrm)
{
    for (size_t k = 0; k < 4 * (size_t)W * H; ++k) vtx[k] = nrm[k] = 0.0f;
    if (n < 1) return 0;
    const float fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3];
    const orc_scene *s0 = S[0];
    const float vs = s0->voxel_size;
    const float inv_s = (float)(1.0 / (double)vs);
    const float B = 8.0f * vs;
    const float mu = s0->mu;
    const int max_iter = (int)(4.0f * (s0->z_max - s0->z_min) / vs) + 64;
    int hits = 0;
#pragma omp parallel for reduction(+ : hits) schedule(dynamic, 2)
    for (int v = 0; v < H; ++v) {
        for (int u = 0; u < W; ++u) {
            size_t o4 = 4 * ((size_t)v * W + u);
            float dc0 = ((float)u - cx) / fx;
            float dc1 = ((float)v - cy) / fy;
            float len = sqrtf((dc0 * dc0 + dc1 * dc1) + 1.0f);
            float dir[3], org[3];
            for (int i = 0; i < 3; ++i) {
                dir[i] = (T_wc[4 * i] * dc0 + T_wc[4 * i + 1] * dc1) + T_wc[4 * i + 2];
                org[i] = T_wc[4 * i + 3];
            }
            const float tB = B / len, tmu = mu / len, ts = vs / len;
            float t = s0->z_min;
            int state = SEARCH_BLOCK_COARSE;
            float X[3];
            for (int it = 0; it < max_iter && t <= s0->z_max; ++it) {
                for (int i = 0; i < 3; ++i) X[i] = org[i] + t * dir[i];
                int alloc = combined_alloc(S, P, n, X, inv_s);
                if (state == SEARCH_BLOCK_COARSE) {
                    if (!alloc) {
                        t = t + tB;
                    } else {
                        t = t - tB;
                        state = SEARCH_BLOCK_FINE;
                    }
                    continue;
                }
                if (!alloc) {
                    if (state == SEARCH_BLOCK_FINE) t = t + tmu;
                    else state = SEARCH_BLOCK_COARSE;
                    continue;
                }
                float F = orc_combined_value(S, P, n, X, NULL);
                if (state == SEARCH_BLOCK_FINE) {
                    if (F <= 0.0f) {
                        state = WRONG_SIDE;
                        break;
                    }
                    state = SEARCH_SURFACE;
                }
                if (F <= 0.0f) {
                    state = BEHIND_SURFACE;
                    break;
                }
                float step = F * tmu;
                if (step < ts) step = ts;
                t = t + step;
            }
            if (state != BEHIND_SURFACE) continue;
            for (int r = 0; r < 2; ++r) {
                for (int i = 0; i < 3; ++i) X[i] = org[i] + t * dir[i];
                float F = orc_combined_value(S, P, n, X, NULL);
                t = t + F * tmu;
            }
            for (int i = 0; i < 3; ++i) X[i] = org[i] + t * dir[i];
            vtx[o4] = X[0];
            vtx[o4 + 1] = X[1];
            vtx[o4 + 2] = X[2];
            vtx[o4 + 3] = 1.0f;
            ++hits;
            float g[3];
            int obs = 1;
            for (int a = 0; a < 3; ++a) {
                float Xp[3] = {X[0], X[1], X[2]}, Xm[3] = {X[0], X[1], X[2]};
                Xp[a] = X[a] + vs;
                Xm[a] = X[a] - vs;
                float dp, dm;
                float fp = orc_combined_value(S, P, n, Xp, &dp);
                float fm = orc_combined_value(S, P, n, Xm, &dm);
                obs &= dp > 0.0f && dm > 0.0f;
                g[a] = fp - fm;
            }
            float gl = sqrtf((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]);
            if (obs && gl > 0.0f) {
                nrm[o4] = g[0] / gl;
                nrm[o4 + 1] = g[1] / gl;
                nrm[o4 + 2] = g[2] / gl;
                nrm[o4 + 3] = 1.0f;
            }
        }
    }
    return hits;
}

/* Test helper: block (bx, by, bz) allocated if missing, its 512 voxels set
 * to sdf / w (index x + 8y + 64z).  Returns 0, or -1 when the block could not
 * be allocated. */
int orc_set_block(orc_scene *s, int bx, int by, int bz, const float *sdf, const float *w)
{
    insert_if_missing(s, bx, by, bz);
    int ptr = lookup(s, bx, by, bz);
    if (ptr < 0) return -1;
    for (int i = 0; i < ORC_BLOCK3; ++i) {
        s->sdf[(size_t)ptr * ORC_BLOCK3 + i] = sdf[i];
        s->w[(size_t)ptr * ORC_BLOCK3 + i] = w[i];
    }
    return 0;
}

/* ---------------------------------------------------------------- swapping */

/* Sec. 5 swapping.  Readings (the section describes the design, not every
 * rule):
 *   - the host map is a block store with one slot per hash entry (O2); a
 *     swapped-out block keeps its entry, marked ptr -1, so a lookup that
 *     meets it sees "not in device memory";
 *   - swap-in is triggered by the allocation: when a segment meets a key
 *     whose entry is swapped out, the entry gets a fresh device block at once
 *     (the device goes on integrating live depth there, O3) and its host data
 *     waits to be fused in (ORC_SW_MERGE);
 *   - orc_swap_in fuses up to K waiting blocks into their device blocks, the
 *     secondary integration of O3: per voxel the weighted mean
 *     (W_d F_d + W_h F_h) / (W_d + W_h) with the weight min(W_d + W_h, max_w),
 *     each operation rounded on its own, the device side first as in the
 *     integration; a voxel the host never observed (W_h = 0) keeps the device
 *     value, one the device has not observed yet (W_d = 0) takes the host
 *     value unchanged;
 *   - orc_swap_out moves up to K blocks to their host slots: blocks in device
 *     memory with no host data waiting whose key no allocation segment has
 *     met for `idle` allocations (the blocks the depth camera no longer
 *     updates); their device blocks return to the free list;
 *   - both take their K blocks in ascending bucket order and, within a
 *     bucket's chain, ascending key (x, y, z as unsigned 16-bit fields, z
 *     most significant): an order that depends only on the set of keys;
 *   - transfers are bounded by K blocks per call (O1). */
int orc_swap_enable(orc_scene *s, int k, int idle)
{
    if (s->swap_on || k <= 0 || idle < 0) return -1;
    const int n = s->nb + s->ne;
    s->swap_state = (uint8_t *)calloc((size_t)n, 1);
    s->touch = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    s->host = (float **)calloc((size_t)n, sizeof(float *));
    s->swap_k = k;
    s->swap_idle = idle;
    s->frame = 0;
    s->swap_on = 1;
    return 0;
}

static uint64_t packed_key(const orc_entry *e)
{
    return (uint64_t)(uint16_t)e->x | ((uint64_t)(uint16_t)e->y << 16) | ((uint64_t)(uint16_t)e->z << 32);
}

static int wants_out(const orc_scene *s, int idx)
{
    const orc_entry *e = &s->entries[idx];
    return e->ptr >= 0 && s->swap_state[idx] == ORC_SW_DEVICE && s->frame - s->touch[idx] >= s->swap_idle;
}

static int wants_in(const orc_scene *s, int idx) { return s->swap_state[idx] == ORC_SW_MERGE; }

/* Up to cap entry indices satisfying pred, bucket by bucket, each chain's in
 * ascending key order. */
static int select_entries(const orc_scene *s, int (*pred)(const orc_scene *, int), int32_t *out, int cap)
{
    int n = 0;
    int32_t *chain = (int32_t *)malloc(sizeof(int32_t) * (size_t)(s->ne + 1));
    for (int h = 0; h < s->nb && n < cap; ++h) {
        if (s->entries[h].ptr < -1) continue; /* bucket never used: no chain */
        int m = 0, idx = h;
        for (;;) {
            if (pred(s, idx)) {
                int j = m++;
                while (j > 0 && packed_key(&s->entries[chain[j - 1]]) > packed_key(&s->entries[idx])) {
                    chain[j] = chain[j - 1];
                    --j;
                }
                chain[j] = idx;
            }
            if (s->entries[idx].offset < 1) break;
            idx = s->nb + s->entries[idx].offset - 1;
        }
        for (int j = 0; j < m && n < cap; ++j) out[n++] = chain[j];
    }
    free(chain);
    return n;
}

/* Moves up to K blocks to the host; returns how many. */
int orc_swap_out(orc_scene *s)
{
    if (!s->swap_on) return -1;
    int32_t *sel = (int32_t *)malloc(sizeof(int32_t) * (size_t)s->swap_k);
    const int n = select_entries(s, wants_out, sel, s->swap_k);
    for (int j = 0; j < n; ++j) {
        const int idx = sel[j];
        orc_entry *e = &s->entries[idx];
        const int ptr = e->ptr;
        if (!s->host[idx]) s->host[idx] = (float *)malloc(sizeof(float) * 2 * ORC_BLOCK3);
        memcpy(s->host[idx], &s->sdf[(size_t)ptr * ORC_BLOCK3], sizeof(float) * ORC_BLOCK3);
        memcpy(s->host[idx] + ORC_BLOCK3, &s->w[(size_t)ptr * ORC_BLOCK3], sizeof(float) * ORC_BLOCK3);
        e->ptr = -1;
        s->swap_state[idx] = ORC_SW_HOST;
        /* the block leaves the allocated list and returns to the free stack */
        int k = 0;
        while (k < s->n_alloc && s->alloc_order[k] != ptr) ++k;
        for (; k + 1 < s->n_alloc; ++k) s->alloc_order[k] = s->alloc_order[k + 1];
        --s->n_alloc;
        s->block_free[s->block_top++] = ptr;
    }
    free(sel);
    s->swapped_out += n;
    return n;
}

/* Secondary fusion of one voxel: device (F, W) and host (Fh, Wh). */
static void fuse_voxel(float *F, float *W, float Fh, float Wh, float max_w)
{
    if (!(Wh > 0.0f)) return;
    if (!(*W > 0.0f)) {
        *F = Fh;
        *W = Wh;
        return;
    }
    float num = *W * *F + Wh * Fh;
    float den = *W + Wh;
    *F = num / den;
    *W = den < max_w ? den : max_w;
}

/* Fuses up to K waiting host blocks into their device blocks; returns how many. */
int orc_swap_in(orc_scene *s)
{
    if (!s->swap_on) return -1;
    int32_t *sel = (int32_t *)malloc(sizeof(int32_t) * (size_t)s->swap_k);
    const int n = select_entries(s, wants_in, sel, s->swap_k);
    const float max_w = (float)s->max_w;
    for (int j = 0; j < n; ++j) {
        const int idx = sel[j];
        const int ptr = s->entries[idx].ptr;
        const float *h = s->host[idx];
        for (int i = 0; i < ORC_BLOCK3; ++i)
            fuse_voxel(&s->sdf[(size_t)ptr * ORC_BLOCK3 + i], &s->w[(size_t)ptr * ORC_BLOCK3 + i], h[i],
                       h[ORC_BLOCK3 + i], max_w);
        s->swap_state[idx] = ORC_SW_DEVICE;
    }
    free(sel);
    s->swapped_in += n;
    return n;
}

/* out: blocks with host data (swapped out or waiting), swapped-out blocks,
 * blocks waiting, blocks moved in, blocks moved out. */
void orc_swap_counters(const orc_scene *s, long long out[5])
{
    long long host = 0, waiting = 0;
    for (int i = 0; s->swap_on && i < s->nb + s->ne; ++i) {
        host += s->swap_state[i] == ORC_SW_HOST;
        waiting += s->swap_state[i] == ORC_SW_MERGE;
    }
    out[0] = host + waiting;
    out[1] = host;
    out[2] = waiting;
    out[3] = s->swapped_in;
    out[4] = s->swapped_out;
}

/* The host slots of the blocks that have host data (swapped out or waiting):
 * coords, sdf, weights and state (ORC_SW_HOST or ORC_SW_MERGE), in entry
 * order; returns the count (all of it when cap is 0 and the arrays NULL). */
int orc_swap_export_host(const orc_scene *s, int16_t *coords, float *sdf, float *w, int32_t *state, int cap)
{
    int n = 0;
    for (int i = 0; s->swap_on && i < s->nb + s->ne; ++i) {
        if (s->swap_state[i] == ORC_SW_DEVICE) continue;
        if (n < cap) {
            coords[3 * n] = s->entries[i].x;
            coords[3 * n + 1] = s->entries[i].y;
            coords[3 * n + 2] = s->entries[i].z;
            memcpy(&sdf[(size_t)n * ORC_BLOCK3], s->host[i], sizeof(float) * ORC_BLOCK3);
            memcpy(&w[(size_t)n * ORC_BLOCK3], s->host[i] + ORC_BLOCK3, sizeof(float) * ORC_BLOCK3);
            state[n] = s->swap_state[i];
        }
        ++n;
    }
    return n;
}

/* ---------------------------------------------------------------- tracking */

/* One level of the depth pyramid (Sec. 4.1.1: "a resolution hierarchy of
 * the depth image").  Output pixel (i, j) of floor(W/2) x floor(H/2) is the
 * mean of the valid (> 0) depths among input pixels (2i, 2j), (2i+1, 2j),
 * (2i, 2j+1), (2i+1, 2j+1), summed in that order and divided by their count;
 * 0 when none is valid. */
void orc_depth_halve(const float *in, int W, int H, float *out)
{
    const int w = W / 2, h = H / 2;
    for (int j = 0; j < h; ++j) {
        for (int i = 0; i < w; ++i) {
            float sum = 0.0f;
            int n = 0;
            for (int k = 0; k < 4; ++k) {
                float d = in[(size_t)(2 * j + (k >> 1)) * W + 2 * i + (k & 1)];
                if (d > 0.0f) {
                    sum = sum + d;
                    ++n;
                }
            }
            out[(size_t)j * w + i] = n > 0 ? sum / (float)n : 0.0f;
        }
    }
}

/*
 * Sec. 4.1.1 ITMDepthTracker, one evaluation: for each depth pixel p (camera
 * point d * ((u-cx)/fx, (v-cy)/fy, 1)) mapped to the world by the current
 * estimate T_g, the projection into the reference view (pose T_ref,
 * intrinsics intr_r, the raycast maps V and N, world coordinates) picks the
 * nearest pixel; with both maps valid there and |T_g p - V| <= dist_thresh,
 * the point-to-plane distance r = (T_g p - V) . N and its derivative with
 * respect to a small world-frame motion (omega, tau) applied to T_g,
 * J = (T_g p x N, N), enter the sums.  Per-pixel arithmetic is float, each
 * operation rounded on its own in the order written; the sums are double.
 * sums[0..20]: sum J_i J_j (i <= j, row-major upper triangle), sums[21..26]:
 * sum J_i r, sums[27]: sum r^2, sums[28]: the number of pixels used.
 * abs_sums (nullable) receives the same sums of absolute values (28).
 */
void orc_icp_reduce(const float *depth, int W, int H, const float intr[4], const float T_g[16], const float *V,
                    const float *N, int Wr, int Hr, const float intr_r[4], const float T_ref[16], float dist_thresh,
                    double *sums, double *abs_sums)
{
    float M[16];
    rigid_inverse(T_ref, M);
    const float t2 = dist_thresh * dist_thresh;
    for (int k = 0; k < 29; ++k) sums[k] = 0.0;
    if (abs_sums)
        for (int k = 0; k < 28; ++k) abs_sums[k] = 0.0;
    for (int v = 0; v < H; ++v) {
        for (int u = 0; u < W; ++u) {
            const float d = depth[(size_t)v * W + u];
            if (!(d > 0.0f)) continue;
            const float pc[3] = {((float)u - intr[2]) / intr[0] * d, ((float)v - intr[3]) / intr[1] * d, d};
            float pw[3], pr[3];
            for (int r = 0; r < 3; ++r) pw[r] = row_apply(T_g + 4 * r, pc[0], pc[1], pc[2]);
            for (int r = 0; r < 3; ++r) pr[r] = row_apply(M + 4 * r, pw[0], pw[1], pw[2]);
            if (!(pr[2] > 0.0f)) continue;
            const float ur = (intr_r[0] * pr[0]) / pr[2] + intr_r[2];
            const float vr = (intr_r[1] * pr[1]) / pr[2] + intr_r[3];
            if (!(ur >= 0.0f && ur <= (float)(Wr - 1) && vr >= 0.0f && vr <= (float)(Hr - 1))) continue;
            const size_t o = 4 * ((size_t)(int)(vr + 0.5f) * Wr + (int)(ur + 0.5f));
            const float *Vp = V + o, *Np = N + o;
            if (!(Vp[3] > 0.0f && Np[3] > 0.0f)) continue;
            const float dx = pw[0] - Vp[0], dy = pw[1] - Vp[1], dz = pw[2] - Vp[2];
            const float dist2 = (dx * dx + dy * dy) + dz * dz;
            if (!(dist2 <= t2)) continue;
            const float res = (dx * Np[0] + dy * Np[1]) + dz * Np[2];
            const float J[6] = {pw[1] * Np[2] - pw[2] * Np[1], pw[2] * Np[0] - pw[0] * Np[2],
                                pw[0] * Np[1] - pw[1] * Np[0], Np[0], Np[1], Np[2]};
            int k = 0;
            for (int i = 0; i < 6; ++i) {
                for (int j = i; j < 6; ++j, ++k) {
                    sums[k] += (double)J[i] * (double)J[j];
                    if (abs_sums) abs_sums[k] += fabs((double)J[i] * (double)J[j]);
                }
            }
            for (int i = 0; i < 6; ++i) {
                sums[21 + i] += (double)J[i] * (double)res;
                if (abs_sums) abs_sums[21 + i] += fabs((double)J[i] * (double)res);
            }
            sums[27] += (double)res * (double)res;
            if (abs_sums) abs_sums[27] += (double)res * (double)res;
            sums[28] += 1.0;
        }
    }
}

/*
 * Gauss-Newton step from the sums (the host side of the tracker): solve
 * H x = -g (H = sum J J^T, g = sum J r) by Cholesky in double, then apply the
 * motion x = (omega, tau) on the world side: T <- [R(omega) | tau] T with
 * R(omega) the rotation by |omega| about omega / |omega| (Rodrigues), in
 * double, rounded to float once.  Returns 0, or -1 (T unchanged) when H is
 * not positive definite.  x (nullable) receives the step.
 */
int orc_icp_update(const double *sums, float T[16], double *x_out)
{
    double A[6][6], b[6];
    int k = 0;
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j, ++k) A[i][j] = A[j][i] = sums[k];
    for (int i = 0; i < 6; ++i) b[i] = -sums[21 + i];
    double L[6][6] = {{0}};
    for (int i = 0; i < 6; ++i) {
        for (int j = 0; j <= i; ++j) {
            double acc = A[i][j];
            for (int m = 0; m < j; ++m) acc -= L[i][m] * L[j][m];
            if (i == j) {
                if (!(acc > 0.0)) return -1;
                L[i][i] = sqrt(acc);
            } else {
                L[i][j] = acc / L[j][j];
            }
        }
    }
    double y[6], x[6];
    for (int i = 0; i < 6; ++i) {
        double acc = b[i];
        for (int m = 0; m < i; ++m) acc -= L[i][m] * y[m];
        y[i] = acc / L[i][i];
    }
    for (int i = 5; i >= 0; --i) {
        double acc = y[i];
        for (int m = i + 1; m < 6; ++m) acc -= L[m][i] * x[m];
        x[i] = acc / L[i][i];
    }
    if (x_out)
        for (int i = 0; i < 6; ++i) x_out[i] = x[i];
    const double th = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    const double K[3][3] = {{0.0, -x[2], x[1]}, {x[2], 0.0, -x[0]}, {-x[1], x[0], 0.0}};
    double K2[3][3], R[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            K2[i][j] = 0.0;
            for (int m = 0; m < 3; ++m) K2[i][j] += K[i][m] * K[m][j];
        }
    const double a = th > 1e-12 ? sin(th) / th : 1.0;
    const double c = th > 1e-12 ? (1.0 - cos(th)) / (th * th) : 0.5;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[i][j] = (i == j ? 1.0 : 0.0) + a * K[i][j] + c * K2[i][j];
    double out[12];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int m = 0; m < 3; ++m) acc += R[i][m] * (double)T[4 * m + j];
            out[4 * i + j] = acc;
        }
        double acc = x[3 + i];
        for (int m = 0; m < 3; ++m) acc += R[i][m] * (double)T[4 * m + 3];
        out[4 * i + 3] = acc;
    }
    for (int i = 0; i < 12; ++i) T[i] = (float)out[i];
    T[12] = T[13] = T[14] = 0.0f;
    T[15] = 1.0f;
    return 0;
}

/* Intrinsics of the next pyramid level: pixel i covers pixels 2i, 2i+1, so
 * the focal lengths halve and the centre maps as c -> (c - 0.5) / 2. */
static void halve_intr(const float in[4], float out[4])
{
    out[0] = in[0] / 2.0f;
    out[1] = in[1] / 2.0f;
    out[2] = (in[2] - 0.5f) / 2.0f;
    out[3] = (in[3] - 0.5f) / 2.0f;
}

/*
 * Coarse-to-fine tracking (Sec. 4.1.1): levels 0 (the input) .. L-1 of the
 * pyramid; from level L-1 down to 0, iters[l] Gauss-Newton steps with
 * outlier distance thresh[l].  A level stops early when fewer than 6 pixels
 * are used or the step cannot be solved.  T (in/out) is the camera-to-world
 * estimate.  Returns the number of steps applied.
 */
int orc_track(const float *depth, int W, int H, const float intr[4], int L, const int *iters, const float *thresh,
              const float *V, const float *N, int Wr, int Hr, const float intr_r[4], const float T_ref[16], float T[16])
{
    float *lev[8];
    int lw[8], lh[8];
    float li[8][4];
    if (L < 1 || L > 8) return 0;
    lev[0] = (float *)depth;
    lw[0] = W;
    lh[0] = H;
    for (int k = 0; k < 4; ++k) li[0][k] = intr[k];
    for (int l = 1; l < L; ++l) {
        lw[l] = lw[l - 1] / 2;
        lh[l] = lh[l - 1] / 2;
        lev[l] = (float *)malloc(sizeof(float) * (size_t)(lw[l] > 0 ? lw[l] : 1) * (size_t)(lh[l] > 0 ? lh[l] : 1));
        orc_depth_halve(lev[l - 1], lw[l - 1], lh[l - 1], lev[l]);
        halve_intr(li[l - 1], li[l]);
    }
    int steps = 0;
    double sums[29];
    for (int l = L - 1; l >= 0; --l) {
        for (int it = 0; it < iters[l]; ++it) {
            orc_icp_reduce(lev[l], lw[l], lh[l], li[l], T, V, N, Wr, Hr, intr_r, T_ref, thresh[l], sums, NULL);
            if (sums[28] < 6.0) break;
            if (orc_icp_update(sums, T, NULL) != 0) break;
            ++steps;
        }
    }
    for (int l = 1; l < L; ++l) free(lev[l]);
    return steps;
}

/* ----------------------------------------------------------------- meshing */

/*
 * Marching Cubes (Sec. 4: "mesh generation via the Marching-Cubes
 * algorithm", Lorensen & Cline 1987) over the zero level set of the TSDF.
 * The triangulation of a cell is derived here from first principles at run
 * time, without a case table: on each of the cube's six faces the crossing
 * points of its sign-changing edges are joined into directed segments (the
 * inside, F < 0, on the segment's left seen from outside the cube); a face
 * with four crossings (diagonal corners inside) joins each crossing to the
 * one across the nearer inside corner, i.e. the inside corners are kept
 * apart.  That choice depends only on the face's four values, so two cells
 * sharing a face agree and the mesh is closed.  The segments chain into
 * closed loops around the cube, each fanned into triangles from its crossing
 * on the lowest-numbered edge, counter-clockwise seen from the outside
 * (F > 0).  Edge 4 a + o1 + 2 o2 runs along axis a from the corner whose
 * other two coordinates are o1 (the lower axis) and o2 (the higher).
 *
 * Corner k of the cell at voxel g sits at g + (k & 1, (k >> 1) & 1, k >> 2).
 * The crossing on the edge from corner a to corner b (b = a + one axis step)
 * is at t = F_a / (F_a - F_b) along that axis: position ((float)g_axis + t) * s
 * on that axis and (float)g * s on the others.
 */

/* the cube's faces: four corners in counter-clockwise order seen from
 * outside (outward normals -x, +x, -y, +y, -z, +z) */
static const int FACE_CORNERS[6][4] = {
    {0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4}, {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6},
};

/* index 0..11 of the edge between corners a and b (differing in one bit) */
static int edge_index(int a, int b)
{
    int lo = a < b ? a : b, hi = a < b ? b : a;
    int axis = (hi - lo) == 1 ? 0 : (hi - lo) == 2 ? 1 : 2;
    /* the 4 edges along an axis are indexed by the other two bits of lo */
    int o1, o2;
    if (axis == 0) {
        o1 = (lo >> 1) & 1;
        o2 = (lo >> 2) & 1;
    } else if (axis == 1) {
        o1 = lo & 1;
        o2 = (lo >> 2) & 1;
    } else {
        o1 = lo & 1;
        o2 = (lo >> 1) & 1;
    }
    return 4 * axis + o1 + 2 * o2;
}

/* Triangles of one cell with corner values F[8] (inside: F < 0); tri
 * receives edge indices, 3 per triangle.  Returns the triangle count. */
static int cell_triangles(const float F[8], int *tri)
{
    int seg_from[12], seg_to[12], n_seg = 0;
    for (int f = 0; f < 6; ++f) {
        const int *q = FACE_CORNERS[f];
        int A[2], B[2], nA = 0, nB = 0, posA[2], posB[2];
        for (int i = 0; i < 4; ++i) {
            int a = q[i], b = q[(i + 1) & 3];
            int ia = F[a] < 0.0f, ib = F[b] < 0.0f;
            if (ia == ib) continue;
            if (ia) { /* inside -> outside along the counter-clockwise walk */
                posA[nA] = i;
                A[nA++] = edge_index(a, b);
            } else {
                posB[nB] = i;
                B[nB++] = edge_index(a, b);
            }
        }
        if (nA == 1) {
            seg_from[n_seg] = A[0];
            seg_to[n_seg++] = B[0];
        } else if (nA == 2) {
            /* diagonal inside corners: the exit crossing on edge i goes to the
             * entry crossing on edge i - 1, around the inside corner q[i] */
            for (int k = 0; k < 2; ++k) {
                int want = (posA[k] + 3) & 3;
                int j = posB[0] == want ? 0 : 1;
                seg_from[n_seg] = A[k];
                seg_to[n_seg++] = B[j];
            }
        }
    }
    int used[12] = {0}, n_tri = 0;
    for (int s0 = 0; s0 < n_seg; ++s0) {
        if (used[s0]) continue;
        int loop[12], n = 0, cur = s0;
        for (int guard = 0; guard < 12; ++guard) {
            used[cur] = 1;
            loop[n++] = seg_from[cur];
            int next = -1;
            for (int t = 0; t < n_seg; ++t)
                if (!used[t] && seg_from[t] == seg_to[cur]) next = t;
            if (next < 0) break;
            cur = next;
        }
        /* fan from the crossing on the lowest-numbered edge (a rule that
         * does not depend on how the loop was found) */
        int first = 0;
        for (int i = 1; i < n; ++i)
            if (loop[i] < loop[first]) first = i;
        int rot[12];
        for (int i = 0; i < n; ++i) rot[i] = loop[(first + i) % n];
        for (int i = 0; i < n; ++i) loop[i] = rot[i];
        /* the loop runs clockwise seen from outside the surface (F > 0):
         * fan it the other way so the triangles face the outside */
        for (int i = 1; i + 1 < n; ++i) {
            tri[3 * n_tri] = loop[0];
            tri[3 * n_tri + 1] = loop[i + 1];
            tri[3 * n_tri + 2] = loop[i];
            ++n_tri;
        }
    }
    return n_tri;
}

static void edge_corners(int e, int *a, int *b)
{
    int axis = e / 4, o = e % 4;
    int o1 = o & 1, o2 = o >> 1;
    int lo;
    if (axis == 0) lo = (o1 << 1) | (o2 << 2);
    else if (axis == 1) lo = o1 | (o2 << 2);
    else lo = o1 | (o2 << 1);
    *a = lo;
    *b = lo | (1 << axis);
}

/* Observed value of voxel g, or 0 when unallocated or never observed. */
static int observed_value(const orc_scene *s, int gx, int gy, int gz, float *F)
{
    int ptr = lookup(s, gx >> 3, gy >> 3, gz >> 3);
    if (ptr < 0) return 0;
    size_t i = (size_t)ptr * ORC_BLOCK3 + (gx & 7) + 8 * (gy & 7) + 64 * (gz & 7);
    if (!(s->w[i] > 0.0f)) return 0;
    *F = s->sdf[i];
    return 1;
}

/* Mesh of the scene: every cell whose 8 corner voxels are allocated and
 * observed, cells visited block by block in allocation order.  Writes up to
 * cap triangles (9 floats each: three world-space vertices) and returns the
 * total count. */
long long orc_mesh(const orc_scene *s, float *out, long long cap)
{
    const float vs = s->voxel_size;
    long long n = 0;
    for (int b = 0; b < s->n_alloc; ++b) {
        int ptr = s->alloc_order[b];
        int bx = s->block_pos[3 * ptr], by = s->block_pos[3 * ptr + 1], bz = s->block_pos[3 * ptr + 2];
        for (int l = 0; l < ORC_BLOCK3; ++l) {
            int g[3] = {8 * bx + (l & 7), 8 * by + ((l >> 3) & 7), 8 * bz + (l >> 6)};
            float F[8];
            int ok = 1;
            for (int k = 0; k < 8 && ok; ++k)
                ok = observed_value(s, g[0] + (k & 1), g[1] + ((k >> 1) & 1), g[2] + (k >> 2), &F[k]);
            if (!ok) continue;
            int tri[36];
            int nt = cell_triangles(F, tri);
            for (int t = 0; t < nt; ++t, ++n) {
                if (n >= cap) continue;
                for (int v = 0; v < 3; ++v) {
                    int a, c;
                    edge_corners(tri[3 * t + v], &a, &c);
                    int axis = (c - a) == 1 ? 0 : (c - a) == 2 ? 1 : 2;
                    float tt = F[a] / (F[a] - F[c]);
                    for (int k = 0; k < 3; ++k) {
                        float coord = (float)(g[k] + ((a >> k) & 1));
                        if (k == axis) coord = coord + tt;
                        out[9 * n + 3 * v + k] = coord * vs;
                    }
                }
            }
        }
    }
    return n;
}

/* Triangles (as edge indices) of a single cell with corner values F[8]:
 * for tests of the triangulation itself.  tri: int[36].  Returns the count. */
int orc_cell_triangles(const float *F, int *tri) { return cell_triangles(F, tri); }

/* ---------------------------------------------------------- introspection */

int orc_status(const orc_scene *s) { return s->status; }
int orc_num_allocated(const orc_scene *s) { return s->n_alloc; }
int orc_excess_used(const orc_scene *s) { return s->ne - s->excess_top; }

/* Copies out the allocated blocks in allocation order: coords (3 x int16),
 * sdf and weight (512 floats each, voxel index x + 8y + 64z). */
int orc_export(const orc_scene *s, int16_t *coords, float *sdf, float *w, int cap)
{
    int n = s->n_alloc < cap ? s->n_alloc : cap;
    for (int k = 0; k < n; ++k) {
        int ptr = s->alloc_order[k];
        memcpy(&coords[3 * k], &s->block_pos[3 * ptr], 3 * sizeof(int16_t));
        if (sdf) memcpy(&sdf[(size_t)k * ORC_BLOCK3], &s->sdf[(size_t)ptr * ORC_BLOCK3], ORC_BLOCK3 * sizeof(float));
        if (w) memcpy(&w[(size_t)k * ORC_BLOCK3], &s->w[(size_t)ptr * ORC_BLOCK3], ORC_BLOCK3 * sizeof(float));
    }
    return n;
}

/* Colour of the allocated blocks in allocation order: coords (3 x int16) and
 * 512 x {r, g, b, colour weight}. */
int orc_export_colour(const orc_scene *s, int16_t *coords, uint8_t *rgbw, int cap)
{
    int n = s->n_alloc < cap ? s->n_alloc : cap;
    for (int k = 0; k < n && s->rgbw; ++k) {
        int ptr = s->alloc_order[k];
        memcpy(&coords[3 * k], &s->block_pos[3 * ptr], 3 * sizeof(int16_t));
        memcpy(&rgbw[(size_t)k * ORC_BLOCK3 * 4], &s->rgbw[(size_t)ptr * ORC_BLOCK3 * 4], ORC_BLOCK3 * 4);
    }
    return n;
}

/* Raw table: per entry x, y, z, offset, ptr as int32. */
void orc_entries(const orc_scene *s, int32_t *out)
{
    for (int i = 0; i < s->nb + s->ne; ++i) {
        out[5 * i + 0] = s->entries[i].x;
        out[5 * i + 1] = s->entries[i].y;
        out[5 * i + 2] = s->entries[i].z;
        out[5 * i + 3] = s->entries[i].offset;
        out[5 * i + 4] = s->entries[i].ptr;
    }
}

/* The depth value of a raw sensor reading in millimetres: raw / 1000,
 * correctly rounded (Sec. 4, view preparation). */
void orc_depth_u16_to_f32(const uint16_t *raw, float *out, long long n)
{
    for (long long i = 0; i < n; ++i) out[i] = (float)raw[i] / 1000.0f;
}

/* ------------------------------------------------ learned confidence weight
 *
 * Not in the paper: a per-pixel observation weight w_px in [0, 1] replaces the
 * constant 1 of the Sec. 4.3 listing.  Readings (all silent in the paper):
 *   features (52): the 7x7 depth patch around the pixel, entry (i, j) for row
 *     offset i and column offset j in -3..3 at index (i+3)*7 + (j+3), equal to
 *     clamp((D(u+j, v+i) - D(u, v)) / mu, -4, 4) when that pixel is inside the
 *     image with depth > 0, else 0; then the unit normal of the back-projected
 *     depth, P(u, v) = D(u, v) ((u-cx)/fx, (v-cy)/fy, 1),
 *     n = normalise((P(u,v+1) - P(u,v-1)) x (P(u+1,v) - P(u-1,v))) (facing the
 *     camera), or 0 when a neighbour is outside or has no depth.
 *   network: h1 = relu(W1 x + b1) (64), h2 = relu(W2 h1 + b2) (64),
 *     o = w3 . h2 + b3, w_px = 1 / (1 + exp(-o)).
 *   parameters (fp32, 7617): W1[64][52], b1[64], W2[64][64], b2[64], w3[64], b3.
 *   with round_bf16, W1, W2 and the inputs of both matrix products (x, h1)
 *     are rounded to bfloat16 (round to nearest even), as the tensor cores
 *     consume them; everything else is fp64 here.
 *   loss: mean binary cross-entropy of w_px against labels y in {0, 1}.
 */

#define ORC_NF 52
#define ORC_NH 64
#define ORC_NP (ORC_NH * ORC_NF + ORC_NH + ORC_NH * ORC_NH + ORC_NH + ORC_NH + 1)

/* bfloat16 round to nearest even of a finite float, returned as float */
float orc_bf16(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

static double depth_at(const float *D, int W, int H, int u, int v)
{
    if (u < 0 || v < 0 || u >= W || v >= H) return 0.0;
    float d = D[(size_t)v * W + u];
    return d > 0.0f ? (double)d : 0.0;
}

/* Features of pixel (u, v); returns 0 (features all zero) when the pixel has
 * no depth. */
int orc_conf_features(const float *D, int W, int H, const float intr[4], float mu, int u, int v, double *x)
{
    for (int k = 0; k < ORC_NF; ++k) x[k] = 0.0;
    double dc = depth_at(D, W, H, u, v);
    if (dc <= 0.0) return 0;
    for (int i = -3; i <= 3; ++i)
        for (int j = -3; j <= 3; ++j) {
            double d = depth_at(D, W, H, u + j, v + i);
            double f = 0.0;
            if (d > 0.0) {
                f = (d - dc) / (double)mu;
                if (f > 4.0) f = 4.0;
                if (f < -4.0) f = -4.0;
            }
            x[(i + 3) * 7 + (j + 3)] = f;
        }
    double dl = depth_at(D, W, H, u - 1, v), dr = depth_at(D, W, H, u + 1, v);
    double du = depth_at(D, W, H, u, v - 1), dd = depth_at(D, W, H, u, v + 1);
    if (dl > 0.0 && dr > 0.0 && du > 0.0 && dd > 0.0) {
        const double fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3];
        double Pl[3] = {dl * ((u - 1) - cx) / fx, dl * (v - cy) / fy, dl};
        double Pr[3] = {dr * ((u + 1) - cx) / fx, dr * (v - cy) / fy, dr};
        double Pu[3] = {du * (u - cx) / fx, du * ((v - 1) - cy) / fy, du};
        double Pd[3] = {dd * (u - cx) / fx, dd * ((v + 1) - cy) / fy, dd};
        double a[3] = {Pd[0] - Pu[0], Pd[1] - Pu[1], Pd[2] - Pu[2]};  /* along +v */
        double b[3] = {Pr[0] - Pl[0], Pr[1] - Pl[1], Pr[2] - Pl[2]};  /* along +u */
        double n[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
        double l = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (l > 0.0) {
            x[49] = n[0] / l;
            x[50] = n[1] / l;
            x[51] = n[2] / l;
        }
    }
    return 1;
}

static double relu(double a) { return a > 0.0 ? a : 0.0; }

static double maybe_bf16(double v, int r) { return r ? (double)orc_bf16((float)v) : v; }

/* Forward pass; returns the logit o.  h1, h2 (nullable) receive the hidden
 * activations, xr (nullable) the inputs as consumed. */
double orc_mlp_forward(const float *P, const double *x, int round_bf16, double *h1, double *h2)
{
    const float *W1 = P, *b1 = W1 + ORC_NH * ORC_NF, *W2 = b1 + ORC_NH, *b2 = W2 + ORC_NH * ORC_NH;
    const float *w3 = b2 + ORC_NH, *b3 = w3 + ORC_NH;
    double xin[ORC_NF], a1[ORC_NH], a1in[ORC_NH], a2[ORC_NH];
    for (int k = 0; k < ORC_NF; ++k) xin[k] = maybe_bf16(x[k], round_bf16);
    for (int m = 0; m < ORC_NH; ++m) {
        double acc = 0.0;
        for (int k = 0; k < ORC_NF; ++k) acc += maybe_bf16(W1[m * ORC_NF + k], round_bf16) * xin[k];
        a1[m] = relu(acc + b1[m]);
        a1in[m] = maybe_bf16(a1[m], round_bf16);
    }
    double o = b3[0];
    for (int n = 0; n < ORC_NH; ++n) {
        double acc = 0.0;
        for (int m = 0; m < ORC_NH; ++m) acc += maybe_bf16(W2[n * ORC_NH + m], round_bf16) * a1in[m];
        a2[n] = relu(acc + b2[n]);
        o += (double)w3[n] * a2[n];
    }
    if (h1)
        for (int m = 0; m < ORC_NH; ++m) h1[m] = a1[m];
    if (h2)
        for (int n = 0; n < ORC_NH; ++n) h2[n] = a2[n];
    return o;
}

/* Mean binary cross-entropy over n samples (X: n x 52, y: n) and its
 * gradient with respect to the 7617 parameters (grad, fp64).  With
 * round_bf16 the forward uses the rounded weights and inputs and the
 * gradient treats the rounding as the identity. */
double orc_mlp_loss_grad(const float *P, const double *X, const float *y, int n, int round_bf16, double *grad)
{
    const float *W1 = P, *b1 = W1 + ORC_NH * ORC_NF, *W2 = b1 + ORC_NH, *b2 = W2 + ORC_NH * ORC_NH;
    const float *w3 = b2 + ORC_NH;
    double *gW1 = grad, *gb1 = gW1 + ORC_NH * ORC_NF, *gW2 = gb1 + ORC_NH, *gb2 = gW2 + ORC_NH * ORC_NH;
    double *gw3 = gb2 + ORC_NH, *gb3 = gw3 + ORC_NH;
    for (int i = 0; i < ORC_NP; ++i) grad[i] = 0.0;
    double loss = 0.0;
    double h1[ORC_NH], h2[ORC_NH], d2[ORC_NH], d1[ORC_NH];
    for (int s = 0; s < n; ++s) {
        const double *x = X + (size_t)s * ORC_NF;
        double o = orc_mlp_forward(P, x, round_bf16, h1, h2);
        double p = 1.0 / (1.0 + exp(-o));
        double t = y[s];
        /* log(1 + exp(-|o|)) form of the cross-entropy */
        loss += (o > 0 ? o : 0.0) - o * t + log1p(exp(-fabs(o)));
        double dout = (p - t) / n;
        gb3[0] += dout;
        for (int k = 0; k < ORC_NH; ++k) {
            gw3[k] += dout * h2[k];
            d2[k] = h2[k] > 0.0 ? dout * w3[k] : 0.0;
            gb2[k] += d2[k];
        }
        for (int a = 0; a < ORC_NH; ++a)
            for (int m = 0; m < ORC_NH; ++m) gW2[a * ORC_NH + m] += d2[a] * maybe_bf16(h1[m], round_bf16);
        for (int m = 0; m < ORC_NH; ++m) {
            double acc = 0.0;
            for (int a = 0; a < ORC_NH; ++a) acc += maybe_bf16(W2[a * ORC_NH + m], round_bf16) * d2[a];
            d1[m] = h1[m] > 0.0 ? acc : 0.0;
            gb1[m] += d1[m];
        }
        for (int m = 0; m < ORC_NH; ++m)
            for (int k = 0; k < ORC_NF; ++k) gW1[m * ORC_NF + k] += d1[m] * maybe_bf16(x[k], round_bf16);
    }
    (void)W1;
    (void)b1;
    (void)b2;
    return loss / n;
}

/* w_px for every pixel of a frame (0 where the pixel has no depth). */
void orc_conf_weights(const float *D, int W, int H, const float intr[4], float mu, const float *P, float *wpx)
{
    double x[ORC_NF];
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            if (!orc_conf_features(D, W, H, intr, mu, u, v, x)) {
                wpx[(size_t)v * W + u] = 0.0f;
                continue;
            }
            double o = orc_mlp_forward(P, x, 1, NULL, NULL);
            wpx[(size_t)v * W + u] = (float)(1.0 / (1.0 + exp(-o)));
        }
}
