// kernels_sort.cu -- stable counting sort of particles by 4x4x4-cell grid
// block, used when particles are loaded into the fused pipeline.  Key of a
// particle: the block containing its stencil base floor(x/dx - 0.5); ties
// keep particle-index order.  Steps: key + histogram, exclusive scan, atomic
// scatter, per-block sort of the (distinct) particle indices so that every
// block lists its particles in index order (the keys array is reused as
// scratch by that last step).
#include "common.cuh"
#include "launch.h"

namespace gbmpm {

// Global block key of particle p: environment * blocks-per-environment + the
// block of its stencil base inside the environment's grid.
__device__ __forceinline__ uint32_t particle_block_key(uint32_t p, float x, float y, float z, const DevParams &P,
                                                       uint32_t &err) {
    int bx, by, bz;
    stencil_axis(x, P.inv_dx, P.n, bx, err);
    stencil_axis(y, P.inv_dx, P.n, by, err);
    stencil_axis(z, P.inv_dx, P.n, bz, err);
    const uint32_t e = P.n_envs > 1 ? env_of_particle(p, P) : 0u;
    return e * P.nbe + block_id(bx >> 2, by >> 2, bz >> 2, P.nb);
}

__global__ void k_keys_hist(DevParams P, const float *__restrict__ x, uint32_t n, uint32_t *__restrict__ keys,
                            uint32_t *__restrict__ counts, Ctrl *ctrl) {
    uint32_t err = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const uint32_t p = base + threadIdx.x;
        const bool ok = p < n;
        uint32_t key = 0xffffffffu;
        if (ok) {
            const float px = x[3 * (size_t)p], py = x[3 * (size_t)p + 1], pz = x[3 * (size_t)p + 2];
            if (!finite3(px, py, pz)) err |= kErrNumeric;
            key = particle_block_key(p, isfinite(px) ? px : 0.f, isfinite(py) ? py : 0.f, isfinite(pz) ? pz : 0.f, P,
                                     err);
            keys[p] = key;
        }
        // one atomic per distinct key in the warp
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(peers) - 1;
        if (ok && (int)(threadIdx.x & 31) == leader) atomicAdd(&counts[key], (uint32_t)__popc(peers));
    }
    if (err) atomicOr(&ctrl->err, err);
}

// Exclusive scan of counts[0..m) into offsets[0..m] and cursor, one CTA.
__global__ void __launch_bounds__(1024) k_scan_counts(const uint32_t *__restrict__ counts, uint32_t m,
                                                      uint32_t *__restrict__ offsets, uint32_t *__restrict__ cursor) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    constexpr int kItems = 4;
    for (uint32_t t0 = 0; t0 < m; t0 += 1024 * kItems) {
        uint32_t v[kItems], sum = 0;
        for (int q = 0; q < kItems; ++q) {
            const uint32_t i = t0 + tid * kItems + q;
            v[q] = i < m ? counts[i] : 0u;
            sum += v[q];
        }
        uint32_t incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = s_warp[lane], wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            s_warp[lane] = wi - w;
        }
        __syncthreads();
        uint32_t run = s_carry + s_warp[warp] + incl - sum;
        for (int q = 0; q < kItems; ++q) {
            const uint32_t i = t0 + tid * kItems + q;
            if (i < m) { offsets[i] = run; cursor[i] = run; }
            run += v[q];
        }
        __syncthreads();
        if (tid == 1023) s_carry = run;
        __syncthreads();
    }
    if (tid == 0) offsets[m] = s_carry;
}

__global__ void k_scatter_ids(const uint32_t *__restrict__ keys, uint32_t n, uint32_t *__restrict__ cursor,
                              uint32_t *__restrict__ perm) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
        perm[atomicAdd(&cursor[keys[p]], 1u)] = p;
}

// Restore index order inside every block's segment of perm (the ids of one
// segment are distinct).  Every chunk of up to kSegSortMax ids is sorted in
// shared memory (bitonic network); a longer segment then merges its sorted
// chunks pairwise, doubling the run length per pass: each id finds its output
// position as its rank in its own run plus the number of smaller ids in the
// partner run (a binary search).  The passes alternate between the segment in
// perm and the same slot range of tmp, so the work is O(c log^2 c) for a
// segment of c ids and no segment reads another's ids.
constexpr int kSegSortMax = 2048;
__global__ void __launch_bounds__(256) k_segment_sort(const uint32_t *__restrict__ offsets, uint32_t m,
                                                      uint32_t *__restrict__ perm, uint32_t *__restrict__ tmp) {
    __shared__ uint32_t s[kSegSortMax];
    const int tid = threadIdx.x;
    for (uint32_t b = blockIdx.x; b < m; b += gridDim.x) {
        const uint32_t off = offsets[b], c = offsets[b + 1] - off;
        if (c <= 1) continue;
        for (uint32_t c0 = 0; c0 < c; c0 += kSegSortMax) {
            const uint32_t cc = min((uint32_t)kSegSortMax, c - c0);
            uint32_t L = 2;
            while (L < cc) L <<= 1;
            for (uint32_t i = tid; i < L; i += blockDim.x) s[i] = i < cc ? perm[off + c0 + i] : 0xffffffffu;
            __syncthreads();
            for (uint32_t k = 2; k <= L; k <<= 1) {
                for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                    for (uint32_t i = tid; i < L; i += blockDim.x) {
                        const uint32_t ixj = i ^ j;
                        if (ixj > i) {
                            const uint32_t a = s[i], bb = s[ixj];
                            const bool up = (i & k) == 0;
                            if ((a > bb) == up) { s[i] = bb; s[ixj] = a; }
                        }
                    }
                    __syncthreads();
                }
            }
            for (uint32_t i = tid; i < cc; i += blockDim.x) perm[off + c0 + i] = s[i];
            __syncthreads();
        }
        if (c <= (uint32_t)kSegSortMax) continue;
        uint32_t *src = perm + off, *dst = tmp + off;
        for (uint32_t w = kSegSortMax; w < c; w <<= 1) {
            for (uint32_t i = tid; i < c; i += blockDim.x) {
                const uint32_t r0 = i / (2 * w) * (2 * w);
                const uint32_t mid = min(r0 + w, c), end = min(r0 + 2 * w, c);
                const uint32_t v = src[i];
                const bool in_a = i < mid;
                // partner run [lo, hi): count its ids smaller than v
                uint32_t lo = in_a ? mid : r0, hi = in_a ? end : mid;
                const uint32_t p0 = lo;
                while (lo < hi) {
                    const uint32_t md = (lo + hi) >> 1;
                    if (src[md] < v) lo = md + 1; else hi = md;
                }
                dst[r0 + (i - (in_a ? r0 : mid)) + (lo - p0)] = v;
            }
            __syncthreads();
            uint32_t *t = src; src = dst; dst = t;
        }
        if (src != perm + off) {
            for (uint32_t i = tid; i < c; i += blockDim.x) perm[off + i] = src[i];
            __syncthreads();
        }
    }
}

void launch_block_sort(const DevParams &P, const float *x, uint32_t n, const SortScratch &s, Ctrl *ctrl, int grid,
                       cudaStream_t st) {
    const uint32_t m = P.nbe * (uint32_t)P.n_envs;
    if (n > 0) k_keys_hist<<<grid, 256, 0, st>>>(P, x, n, s.keys, s.counts, ctrl);
    k_scan_counts<<<1, 1024, 0, st>>>(s.counts, m, s.offsets, s.cursor);
    if (n == 0) return;
    k_scatter_ids<<<grid, 256, 0, st>>>(s.keys, n, s.cursor, s.perm);
    k_segment_sort<<<grid, 256, 0, st>>>(s.offsets, m, s.perm, s.keys);
}

// --------------------------------------------------------- placement

__global__ void k_place_sorted(const float *__restrict__ x, const float *__restrict__ v, const float *__restrict__ F,
                               const float *__restrict__ C, uint32_t n, const uint32_t *__restrict__ perm, PState S,
                               VCState V) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const size_t p = perm[j];
        S.xi[j] = make_float4(x[3 * p], x[3 * p + 1], x[3 * p + 2], __uint_as_float((uint32_t)p));
        float f[9], c[9], vv[3];
        for (int q = 0; q < 9; ++q) {
            f[q] = F ? F[9 * p + q] : ((q % 4) == 0 ? 1.0f : 0.0f);
            c[q] = C ? C[9 * p + q] : 0.0f;
        }
        for (int q = 0; q < 3; ++q) vv[q] = v ? v[3 * p + q] : 0.0f;
        S.f0[j] = make_float4(f[0], f[1], f[2], f[3]);
        S.f1[j] = make_float4(f[4], f[5], f[6], f[7]);
        S.f2[j] = f[8];
        store_vc(V, j, vv[0], vv[1], vv[2], c);
    }
}

void launch_place_sorted(const DevParams &P, const float *x, const float *v, const float *F, const float *C,
                         uint32_t n, const SortScratch &s, const PState &S, const VCState &V, int grid,
                         cudaStream_t st) {
    (void)P;
    if (n == 0) return;
    k_place_sorted<<<grid, 256, 0, st>>>(x, v, F, C, n, s.perm, S, V);
}

// Run tables for sub-step `step`: every non-empty block b is a source with
// one chunk (index b) whose particles all stay in b (direction 13).  Also
// lists b as active and puts its 27 neighbouring grid blocks on the clear
// list of G[step % 3], which the load's P2G writes.
__global__ void k_init_tables(DevParams P, const uint32_t *__restrict__ offsets, FusedBufs B, uint32_t step) {
    const uint32_t m = B.nblocks;
    const int par = step & 1, m3 = step % 3;
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < m; b += gridDim.x * blockDim.x) {
        const uint32_t off = offsets[b], c = offsets[b + 1] - off;
        if (c == 0) continue;
        BlockTab t;
        t.stamp = step; t.first = b; t.npass = 1; t.pad = 0;
        B.tabs[par][b] = t;
        Chunk &ch = B.chunks[par][b];
        for (int d = 0; d < 27; ++d) ch.run[d] = make_uint2(d == 13 ? off : 0u, d == 13 ? c : 0u);
        B.inbox[par][(size_t)b * kInbox + 13 * kNpMax] = make_uint4(off, c, step, 0u);
        B.astamp[b] = step;
        B.alist[par][atomicAdd(&B.ctrl->nactive[par][0], 1u)] = b;
        const uint32_t e = b / P.nbe, bl = b % P.nbe;
        const int bx = bl % P.nb, by = (bl / P.nb) % P.nb, bz = bl / (P.nb * P.nb);
        for (int d = 0; d < 27; ++d) {
            const int sx = bx + d % 3 - 1, sy = by + (d / 3) % 3 - 1, sz = bz + d / 9 - 1;
            if (sx < 0 || sy < 0 || sz < 0 || sx >= P.nb || sy >= P.nb || sz >= P.nb) continue;
            const uint32_t g = e * P.nbe + block_id(sx, sy, sz, P.nb);
            if (atomicExch(&B.gstamp[g], step) != step) B.clist[m3][atomicAdd(&B.ctrl->nclear[m3], 1u)] = g;
        }
    }
}

void launch_init_tables(const DevParams &P, const SortScratch &s, const FusedBufs &B, uint32_t step, int grid,
                        cudaStream_t st) {
    k_init_tables<<<grid, 256, 0, st>>>(P, s.offsets, B, step);
}

}  // namespace gbmpm
