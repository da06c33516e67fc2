// Sec. 4 mesh generation by Marching Cubes (Lorensen & Cline 1987) over the
// zero level set of the TSDF (inside: F < 0).
//
// Cells are the voxel cubes g + {0,1}^3 whose eight corners are allocated
// and observed (weight > 0); cells that straddle blocks read the neighbour
// blocks.  The triangulation of each of the 256 inside/outside corner
// patterns is built once on the host (build_table): the crossings of the
// sign-changing edges are linked face by face, a face with two diagonal
// inside corners separating them (a rule that depends only on the face, so
// neighbouring cells agree and the mesh is closed); the links form loops,
// each oriented by a geometric test and fanned from its crossing on the
// lowest-numbered edge, counter-clockwise seen from outside (F > 0).
// Edge 4 a + o1 + 2 o2 runs along axis a from the corner whose other two
// coordinates are o1 (lower axis) and o2 (higher axis).  A crossing sits at
// t = F_a / (F_a - F_b) from the edge's lower corner: coordinate
// (g + t) * s along the edge's axis, g * s on the others, each operation
// rounded on its own (built with -fmad=false).
//
// One CTA per allocated block (persistent grid-stride): the block's 9x9x9
// voxel neighbourhood (the block and the +1 layers of up to seven
// neighbours, each looked up once) is staged in shared memory with the case
// table; a thread meshes a cell, and a warp reserves its output slots with
// one atomic after a prefix sum over its lanes' triangle counts.
#include "itm_ops.cuh"

namespace itm {

namespace {

struct McTable {
    uint8_t count[256];
    uint8_t edge[256][15];  // 3 edge indices per triangle
};

// Corner k of a cell sits at (k & 1, (k >> 1) & 1, k >> 2); edge e = 4 a + o1 +
// 2 o2 runs along axis a from its lower corner.
int edge_lo(int e)
{
    const int a = e >> 2, o1 = e & 1, o2 = (e >> 1) & 1;
    const int ua = a == 0 ? 1 : 0, va = a == 2 ? 1 : 2;  // the other axes, lower first
    return (o1 << ua) | (o2 << va);
}
int edge_hi(int e) { return edge_lo(e) | (1 << (e >> 2)); }

// The case table, derived as a graph: the crossings (edges with one inside and
// one outside corner) are its nodes, and each face of the cube links the
// crossings on its four sides -- two crossings are linked to each other, four
// (two inside corners on a diagonal) are linked in pairs around each inside
// corner, which separates the diagonal corners (a choice that depends on the
// face alone, so the two cells sharing the face agree and the mesh is closed).
// Every crossing has one link on each of its two faces, so the links form
// loops.  A loop is oriented by geometry: on the face of its first link, seen
// from outside the cube, the inside corner of the first crossing must lie to
// the left of the step from the first crossing's midpoint to the second's
// (inside on the left: the loop runs clockwise seen from the F > 0 side).  It
// is then fanned from its crossing on the lowest-numbered edge, each triangle
// (first, next, current) so that it faces the F > 0 side.
void build_table(McTable &T)
{
    memset(&T, 0, sizeof(T));
    for (int cfg = 0; cfg < 256; ++cfg) {
        auto inside = [cfg](int k) { return ((cfg >> k) & 1) != 0; };
        int link[12][2], face_of[12][2], nl[12] = {0};
        for (int f = 0; f < 6; ++f) {
            const int a = f >> 1, side = f & 1;
            int sides[4], ns = 0;
            for (int e = 0; e < 12; ++e) {
                if ((e >> 2) == a) continue;  // an edge along the face normal is not on the face
                const int lo = edge_lo(e), hi = edge_hi(e);
                if (((lo >> a) & 1) != side) continue;
                if (inside(lo) != inside(hi)) sides[ns++] = e;
            }
            int pairs[2][2], np = 0;
            if (ns == 2) {
                pairs[np][0] = sides[0];
                pairs[np++][1] = sides[1];
            } else if (ns == 4) {
                // pair the two crossings at each inside corner of the face
                for (int i = 0; i < 4; ++i)
                    for (int j = i + 1; j < 4; ++j) {
                        const int c0[2] = {edge_lo(sides[i]), edge_hi(sides[i])};
                        const int c1[2] = {edge_lo(sides[j]), edge_hi(sides[j])};
                        for (int x = 0; x < 2; ++x)
                            for (int y = 0; y < 2; ++y)
                                if (c0[x] == c1[y] && inside(c0[x]) && np < 2) {
                                    pairs[np][0] = sides[i];
                                    pairs[np++][1] = sides[j];
                                }
                    }
            }
            for (int q = 0; q < np; ++q)
                for (int h = 0; h < 2; ++h) {
                    const int e = pairs[q][h];
                    link[e][nl[e]] = pairs[q][1 - h];
                    face_of[e][nl[e]++] = f;
                }
        }
        bool seen[12] = {false};
        int nt = 0;
        for (int e0 = 0; e0 < 12; ++e0) {
            if (nl[e0] != 2 || seen[e0]) continue;
            int loop[12], n = 0, prev = -1, cur = e0;
            do {  // follow the links: each crossing has two, leave by the one not arrived on
                seen[cur] = true;
                loop[n++] = cur;
                const int nxt = link[cur][0] == prev ? link[cur][1] : link[cur][0];
                prev = cur;
                cur = nxt;
            } while (cur != e0 && n < 12);
            // orientation: outward normal of the face linking loop[0] and loop[1]
            const int f = link[loop[0]][0] == loop[1] ? face_of[loop[0]][0] : face_of[loop[0]][1];
            const int a = f >> 1;
            const double nrm = (f & 1) ? 1.0 : -1.0;
            auto mid = [](int e, double *m) {
                const int lo = edge_lo(e), hi = edge_hi(e);
                for (int k = 0; k < 3; ++k) m[k] = 0.5 * (((lo >> k) & 1) + ((hi >> k) & 1));
            };
            double m0[3], m1[3], c[3];
            mid(loop[0], m0);
            mid(loop[1], m1);
            const int in0 = inside(edge_lo(loop[0])) ? edge_lo(loop[0]) : edge_hi(loop[0]);
            for (int k = 0; k < 3; ++k) c[k] = (double)((in0 >> k) & 1);
            const double d[3] = {m1[0] - m0[0], m1[1] - m0[1], m1[2] - m0[2]};
            const double w[3] = {c[0] - m0[0], c[1] - m0[1], c[2] - m0[2]};
            const double cross_a = d[(a + 1) % 3] * w[(a + 2) % 3] - d[(a + 2) % 3] * w[(a + 1) % 3];
            if (cross_a * nrm < 0.0)  // inside corner on the right: reverse the loop
                for (int i = 0, j = n - 1; i < j; ++i, --j) {
                    const int t = loop[i];
                    loop[i] = loop[j];
                    loop[j] = t;
                }
            int first = 0;
            for (int i = 1; i < n; ++i)
                if (loop[i] < loop[first]) first = i;
            for (int i = 1; i + 1 < n; ++i) {
                T.edge[cfg][3 * nt] = (uint8_t)loop[first];
                T.edge[cfg][3 * nt + 1] = (uint8_t)loop[(first + i + 1) % n];
                T.edge[cfg][3 * nt + 2] = (uint8_t)loop[(first + i) % n];
                ++nt;
            }
        }
        T.count[cfg] = (uint8_t)nt;
    }
}

constexpr int kMeshThreads = 256;
constexpr int kHalo = 9;  // a block plus the +1 layers

template <int MODE>
__global__ void __launch_bounds__(kMeshThreads) mesh_kernel(SceneDev s, const McTable tab, float *__restrict__ out,
                                                            long long cap, unsigned long long *__restrict__ counter)
{
    __shared__ McTable st;
    __shared__ float F[kHalo * kHalo * kHalo];
    __shared__ uint8_t ob[kHalo * kHalo * kHalo];
    __shared__ int P[8];
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&tab);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&st);
        for (int i = threadIdx.x; i < (int)(sizeof(McTable) / 4); i += blockDim.x) dst[i] = src[i];
    }
    const int n = min(__ldcg(&s.ctr->block_head), s.nv);
    const int lane = threadIdx.x & 31;
    const float vs = s.voxel_size;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int ptr = __ldg(&s.block_free[i]);
        const short4 b = __ldg(&s.block_pos[ptr]);
        if (!b.w) continue;  // uniform over the CTA
        __syncthreads();     // the previous block's staging is no longer read
        if (threadIdx.x < 8) {
            const int t = threadIdx.x;
            const int bx = b.x + (t & 1), by = b.y + ((t >> 1) & 1), bz = b.z + (t >> 2);
            P[t] = t == 0 ? ptr : (in_i16(bx) && in_i16(by) && in_i16(bz) ? lookup_ro(s, bx, by, bz) : -1);
        }
        __syncthreads();
        for (int v = threadIdx.x; v < kHalo * kHalo * kHalo; v += blockDim.x) {
            const int x = v % kHalo, y = (v / kHalo) % kHalo, z = v / (kHalo * kHalo);
            const int p = P[(x >> 3) | ((y >> 3) << 1) | ((z >> 3) << 2)];
            uint8_t o = 0;
            float f = 1.0f;
            if (p >= 0) {
                const size_t idx = (size_t)p * kBlockVoxels + (x & 7) + 8 * (y & 7) + 64 * (z & 7);
                o = MODE == 0 ? (__ldg(&s.w8[idx]) != 0) : (__ldg(&s.w32[idx]) > 0.0f);
                f = __ldg(&s.sdf[idx]);
            }
            F[v] = f;
            ob[v] = o;
        }
        __syncthreads();
        for (int c = threadIdx.x; c < kBlockVoxels; c += blockDim.x) {  // all lanes take part
            const int cx = c & 7, cy = (c >> 3) & 7, cz = c >> 6;
            float Fc[8];
            bool all = true;
            int cfg = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int v = (cx + (k & 1)) + kHalo * ((cy + ((k >> 1) & 1)) + kHalo * (cz + (k >> 2)));
                all = all && ob[v];
                Fc[k] = F[v];
                cfg |= (Fc[k] < 0.0f ? 1 : 0) << k;
            }
            const int nt = all ? st.count[cfg] : 0;
            // warp prefix sum of the triangle counts, one atomic per warp
            int incl = nt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(kFull, incl, 31);
            unsigned long long base = 0;
            if (lane == 31 && total > 0) base = atomicAdd(counter, (unsigned long long)total);
            base = __shfl_sync(kFull, base, 31);
            const long long first = (long long)base + (incl - nt);
            const int gx = 8 * b.x + cx, gy = 8 * b.y + cy, gz = 8 * b.z + cz;
            for (int t = 0; t < nt; ++t) {
                if (first + t >= cap) break;
                float *o = out + (size_t)(first + t) * 9;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const int e = st.edge[cfg][3 * t + j];
                    const int axis = e >> 2, o1 = e & 1, o2 = (e >> 1) & 1;
                    const int ua = axis == 0 ? 1 : 0, va = axis == 2 ? 1 : 2;
                    const int ka = (o1 << ua) | (o2 << va), kb = ka | (1 << axis);
                    const float tt = fdiv(Fc[ka], fsub(Fc[ka], Fc[kb]));
                    const int g[3] = {gx + (ka & 1), gy + ((ka >> 1) & 1), gz + (ka >> 2)};
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        float coord = (float)g[k];
                        if (k == axis) coord = fadd(coord, tt);
                        o[3 * j + k] = fmul(coord, vs);
                    }
                }
            }
        }
    }
}

// built on first use (a function-local static: thread-safe initialisation)
const McTable &mc_table()
{
    static const McTable T = [] {
        McTable t;
        build_table(t);
        return t;
    }();
    return T;
}

}  // namespace

int mesh_case_table(uint8_t *count, uint8_t *edges)
{
    const McTable &t = mc_table();
    memcpy(count, t.count, sizeof(t.count));
    memcpy(edges, t.edge, sizeof(t.edge));
    return ITM_OK;
}

cudaError_t launch_mesh(const SceneDev &s, float *out, long long cap, unsigned long long *counter, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int g = 4 * (sms > 0 ? sms : 1);
    if (s.weight_mode == 0)
        mesh_kernel<0><<<g, kMeshThreads, 0, st>>>(s, mc_table(), out, cap, counter);
    else
        mesh_kernel<1><<<g, kMeshThreads, 0, st>>>(s, mc_table(), out, cap, counter);
    return cudaGetLastError();
}

}  // namespace itm

extern "C" int itm_mesh_case_table(uint8_t *count, uint8_t *edges)
{
    if (!count || !edges) return ITM_ERR_ARG;
    return itm::mesh_case_table(count, edges);
}
