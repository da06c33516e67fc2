// Sec. 4 mesh generation by Marching Cubes (Lorensen & Cline 1987) over the
// zero level set of the TSDF (inside: F < 0).
//
// Cells are the voxel cubes g + {0,1}^3 whose eight corners are allocated
// and observed (weight > 0); cells that straddle blocks read the neighbour
// blocks.  The triangulation of each of the 256 inside/outside corner
// patterns is built once on the host by walking the cube's faces: on each
// face the crossings of its sign-changing edges are joined into directed
// segments (inside on the left seen from outside the cube), a face with two
// diagonal inside corners cutting off each inside corner (a rule that
// depends only on the face, so neighbouring cells agree and the mesh is
// closed); the segments chain into loops, each fanned from its crossing on
// the lowest-numbered edge, counter-clockwise seen from outside (F > 0).
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

int edge_id(int k1, int k2)
{
    const int d = k1 ^ k2;
    const int axis = d == 1 ? 0 : (d == 2 ? 1 : 2);
    const int lo = k1 < k2 ? k1 : k2;
    const int u = axis == 0 ? 1 : 0, v = axis == 2 ? 1 : 2;  // the other axes, lower first
    return 4 * axis + ((lo >> u) & 1) + 2 * ((lo >> v) & 1);
}

void build_table(McTable &T)
{
    memset(&T, 0, sizeof(T));
    for (int cfg = 0; cfg < 256; ++cfg) {
        int from[12], to[12], ns = 0;
        for (int a = 0; a < 3; ++a) {
            const int u = (a + 1) % 3, v = (a + 2) % 3;  // (u, v, a) right-handed
            for (int side = 0; side < 2; ++side) {
                // corners counter-clockwise seen from outside (normal +a for side 1)
                static const int uv1[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
                static const int uv0[4][2] = {{0, 0}, {0, 1}, {1, 1}, {1, 0}};
                int q[4];
                for (int i = 0; i < 4; ++i) {
                    const int *p = side ? uv1[i] : uv0[i];
                    q[i] = (side << a) | (p[0] << u) | (p[1] << v);
                }
                int exits[2], entries[2], exit_pos[2], entry_pos[2], ne = 0, nn = 0;
                for (int i = 0; i < 4; ++i) {
                    const bool in0 = (cfg >> q[i]) & 1, in1 = (cfg >> q[(i + 1) & 3]) & 1;
                    if (in0 == in1) continue;
                    if (in0) {
                        exit_pos[ne] = i;
                        exits[ne++] = edge_id(q[i], q[(i + 1) & 3]);
                    } else {
                        entry_pos[nn] = i;
                        entries[nn++] = edge_id(q[i], q[(i + 1) & 3]);
                    }
                }
                for (int k = 0; k < ne; ++k) {
                    // the exit on edge i pairs with the entry on edge i - 1
                    // (the two edges at the inside corner q[i])
                    int j = 0;
                    if (ne == 2 && entry_pos[0] != ((exit_pos[k] + 3) & 3)) j = 1;
                    from[ns] = exits[k];
                    to[ns++] = entries[j];
                }
            }
        }
        bool used[12] = {false};
        int nt = 0;
        for (int s0 = 0; s0 < ns; ++s0) {
            if (used[s0]) continue;
            int loop[12], n = 0, cur = s0;
            while (cur >= 0 && !used[cur] && n < 12) {
                used[cur] = true;
                loop[n++] = from[cur];
                int next = -1;
                for (int t = 0; t < ns; ++t)
                    if (!used[t] && from[t] == to[cur]) next = t;
                cur = next;
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
