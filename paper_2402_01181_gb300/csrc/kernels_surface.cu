// kernels_surface.cu -- iso-surface extraction of the grid density, the
// renderer's Marching Cubes step (Sec. III), in its tetrahedral form: every
// cell is split into six tetrahedra around its diagonal from corner 0 to
// corner 7 (corner c at offset (c & 1, (c >> 1) & 1, (c >> 2) & 1)), each of
// which contributes 0, 1 or 2 triangles facing away from the inside
// (density >= iso).  Neighbouring cells split their shared faces alike, so
// the surface is closed.  Three passes: triangle counts per cell, an
// exclusive scan, and the triangles written in cell order (i fastest).
#include "common.cuh"
#include "launch.h"

namespace gbmpm {

namespace {

constexpr int kScanBlock = 1024;

__device__ __forceinline__ void corner_of(int c, int &x, int &y, int &z) {
    x = c & 1;
    y = (c >> 1) & 1;
    z = (c >> 2) & 1;
}

// The six tetrahedra (0, a, b, 7) along the paths 0 -> a -> b -> 7, with
// corners 1 and 2 swapped where needed for a positive orientation (sign of
// det[B - A, C - A, D - A] over the integer corner offsets).
__device__ __forceinline__ void tetrahedron(int q, int t[4]) {
    const int pa[6] = {1, 1, 2, 2, 4, 4}, pb[6] = {3, 5, 3, 6, 5, 6};
    t[0] = 0; t[1] = pa[q]; t[2] = pb[q]; t[3] = 7;
    int u[3], v[3], w[3];
    corner_of(t[1], u[0], u[1], u[2]);
    corner_of(t[2], v[0], v[1], v[2]);
    corner_of(t[3], w[0], w[1], w[2]);
    const int det = u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) +
                    u[2] * (v[0] * w[1] - v[1] * w[0]);
    if (det < 0) { const int x = t[1]; t[1] = t[2]; t[2] = x; }
}

__device__ __forceinline__ int tet_count(const float f[8], float iso, const int t[4]) {
    int nin = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) nin += f[t[q]] >= iso;
    return nin == 2 ? 2 : (nin == 1 || nin == 3 ? 1 : 0);
}

__device__ __forceinline__ void load_cell(const float4 *__restrict__ G, int nb, uint32_t nbe, uint32_t env, int i,
                                          int j, int k, float scale, float f[8]) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        int x, y, z;
        corner_of(c, x, y, z);
        f[c] = __ldg(&G[node_addr_env(env, i + x, j + y, k + z, nb, nbe)].x) * scale;
    }
}

__device__ __forceinline__ void cell_of(uint32_t c, int m, int &i, int &j, int &k) {
    i = (int)(c % (uint32_t)m);
    j = (int)((c / (uint32_t)m) % (uint32_t)m);
    k = (int)(c / ((uint32_t)m * (uint32_t)m));
}

__global__ void __launch_bounds__(256) k_surface_count(const float4 *__restrict__ G, int n, int nb, uint32_t nbe,
                                                        uint32_t env, float scale, float iso, uint32_t *__restrict__ counts) {
    const int m = n - 1;
    const uint32_t cells = (uint32_t)m * m * m;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += gridDim.x * blockDim.x) {
        int i, j, k;
        cell_of(c, m, i, j, k);
        float f[8];
        load_cell(G, nb, nbe, env, i, j, k, scale, f);
        int cnt = 0;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            int t[4];
            tetrahedron(q, t);
            cnt += tet_count(f, iso, t);
        }
        counts[c] = (uint32_t)cnt;
    }
}

// exclusive scan of n counts in place: per-1024 block scans, their totals
// scanned by one CTA, then added back
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *s_warp, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    total = s_warp[32];
    const uint32_t r = s_warp[warp] + incl - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_blocks(uint32_t *__restrict__ a, uint32_t n,
                                                           uint32_t *__restrict__ sums) {
    __shared__ uint32_t s_warp[33];
    const uint32_t i = blockIdx.x * kScanBlock + threadIdx.x;
    const uint32_t v = i < n ? a[i] : 0u;
    uint32_t total;
    const uint32_t e = block_exclusive_scan(v, s_warp, total);
    if (i < n) a[i] = e;
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// one CTA: exclusive scan of the block totals, and the grand total at sums[nblk]
__global__ void __launch_bounds__(kScanBlock) k_scan_sums(uint32_t *__restrict__ sums, uint32_t nblk) {
    __shared__ uint32_t s_warp[33];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < nblk; base += kScanBlock) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < nblk ? sums[i] : 0u;
        uint32_t total;
        const uint32_t e = block_exclusive_scan(v, s_warp, total);
        if (i < nblk) sums[i] = carry + e;
        carry += total;
    }
    if (threadIdx.x == 0) sums[nblk] = carry;
}

__global__ void k_scan_add(uint32_t *__restrict__ a, uint32_t n, const uint32_t *__restrict__ sums) {
    const uint32_t i = blockIdx.x * kScanBlock + threadIdx.x;
    if (i < n) a[i] += sums[blockIdx.x];
}

// point where the density crosses iso on the edge between corners a, b of the
// cell, computed from the lower-numbered corner
__device__ __forceinline__ void edge_point(int i, int j, int k, int a, int b, const float f[8], float iso, float dx,
                                           float *out) {
    if (a > b) { const int x = a; a = b; b = x; }
    int ax, ay, az, bx, by, bz;
    corner_of(a, ax, ay, az);
    corner_of(b, bx, by, bz);
    const float t = (iso - f[a]) / (f[b] - f[a]);
    out[0] = ((float)(i + ax) + t * (float)(bx - ax)) * dx;
    out[1] = ((float)(j + ay) + t * (float)(by - ay)) * dx;
    out[2] = ((float)(k + az) + t * (float)(bz - az)) * dx;
}

__device__ __forceinline__ void put_triangle(float *__restrict__ tri, uint64_t slot, uint64_t max_tri, int i, int j,
                                             int k, const int e[3][2], const float f[8], float iso, float dx) {
    if (slot >= max_tri) return;
    float v[9];
#pragma unroll
    for (int q = 0; q < 3; ++q) edge_point(i, j, k, e[q][0], e[q][1], f, iso, dx, v + 3 * q);
#pragma unroll
    for (int q = 0; q < 9; ++q) tri[9 * slot + q] = v[q];
}

__global__ void __launch_bounds__(256) k_surface_emit(const float4 *__restrict__ G, int n, int nb, uint32_t nbe,
                                                       uint32_t env, float scale, float iso, float dx,
                                                       const uint32_t *__restrict__ offsets, float *__restrict__ tri,
                                                       uint64_t max_tri) {
    const int m = n - 1;
    const uint32_t cells = (uint32_t)m * m * m;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += gridDim.x * blockDim.x) {
        const uint32_t first = offsets[c];
        if (offsets[c + 1] == first) continue;
        int i, j, k;
        cell_of(c, m, i, j, k);
        float f[8];
        load_cell(G, nb, nbe, env, i, j, k, scale, f);
        uint64_t slot = first;
        for (int q = 0; q < 6; ++q) {
            int t[4];
            tetrahedron(q, t);
            int in[4], nin = 0;
#pragma unroll
            for (int r = 0; r < 4; ++r) { in[r] = f[t[r]] >= iso; nin += in[r]; }
            if (nin == 0 || nin == 4) continue;
            if (nin == 1 || nin == 3) {
                // the lone vertex first, in an even permutation of t
                int lone = 0;
                for (int r = 0; r < 4; ++r) if (in[r] == (nin == 1)) lone = r;
                const int perms[4][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {2, 0, 1, 3}, {3, 0, 2, 1}};
                const int *p = perms[lone];
                int e[3][2] = {{t[p[0]], t[p[1]]}, {t[p[0]], t[p[2]]}, {t[p[0]], t[p[3]]}};
                if (nin == 3) {   // the inside is on the other side: reverse
                    const int s0 = e[1][0], s1 = e[1][1];
                    e[1][0] = e[2][0]; e[1][1] = e[2][1]; e[2][0] = s0; e[2][1] = s1;
                }
                put_triangle(tri, slot++, max_tri, i, j, k, e, f, iso, dx);
            } else {
                // inside (p, q), outside (r, s) in an even permutation of t: the
                // quad pr, ps, qs, qr as two triangles
                int perm[4], a = 0, b = 2;
                for (int r = 0; r < 4; ++r) { if (in[r]) perm[a++] = r; else perm[b++] = r; }
                int inv = 0;
                for (int x = 0; x < 4; ++x)
                    for (int y = x + 1; y < 4; ++y) inv += perm[x] > perm[y];
                if (inv & 1) { const int x = perm[2]; perm[2] = perm[3]; perm[3] = x; }
                const int P = t[perm[0]], Q = t[perm[1]], R = t[perm[2]], S = t[perm[3]];
                const int e1[3][2] = {{P, R}, {P, S}, {Q, S}};
                const int e2[3][2] = {{P, R}, {Q, S}, {Q, R}};
                put_triangle(tri, slot++, max_tri, i, j, k, e1, f, iso, dx);
                put_triangle(tri, slot++, max_tri, i, j, k, e2, f, iso, dx);
            }
        }
    }
}

}  // namespace

// counts: (n-1)^3 + 1 entries, sums: ceil(((n-1)^3 + 1) / 1024) + 1 entries.
// On return counts holds the exclusive prefix (its last entry the total).
void launch_surface_count_scan(const float4 *G, int n, int nb, uint32_t nbe, uint32_t env, float scale, float iso,
                               uint32_t *counts, uint32_t *sums, int grid, cudaStream_t st) {
    const uint32_t cells = (uint32_t)(n - 1) * (n - 1) * (n - 1);
    k_surface_count<<<grid, 256, 0, st>>>(G, n, nb, nbe, env, scale, iso, counts);
    cudaMemsetAsync(counts + cells, 0, sizeof(uint32_t), st);
    const uint32_t len = cells + 1, nblk = (len + kScanBlock - 1) / kScanBlock;
    k_scan_blocks<<<nblk, kScanBlock, 0, st>>>(counts, len, sums);
    k_scan_sums<<<1, kScanBlock, 0, st>>>(sums, nblk);
    k_scan_add<<<nblk, kScanBlock, 0, st>>>(counts, len, sums);
}

void launch_surface_emit(const float4 *G, int n, int nb, uint32_t nbe, uint32_t env, float scale, float iso, float dx,
                         const uint32_t *offsets, float *tri, uint64_t max_tri, int grid, cudaStream_t st) {
    k_surface_emit<<<grid, 256, 0, st>>>(G, n, nb, nbe, env, scale, iso, dx, offsets, tri, max_tri);
}

}  // namespace gbmpm
