// kernels_reverse.cu -- reverse mode of the fused sub-step, block by block.
//
// The forward pass of a differentiable rollout on the fused pipeline records,
// for every sub-step k of the segment being reversed, the input particles of
// each occupied 4x4x4-cell block in block-contiguous order and the grid G_k
// the sub-step read.  The reverse sub-step k then runs one CTA per recorded
// block b, mirroring the forward launch:
//   1. the grid operation of G_k over the 6^3 nodes [4b, 4b+5]^3 (Eq. 7,
//      gravity, tools, walls) into a shared tile of velocities V_k, and the
//      adjoint dL/d(m, mv) of G_{k+1} over the 8^3 nodes [4b-1, 4b+6]^3 into
//      a second tile;
//   2. per particle: (x, v, C, F) after sub-step k from the recorded v and C
//      (Eqs. 8-9 as the forward pass evaluated them, then Eqs. 4, 10); the reverse of P2G of sub-step
//      k+1 (Eqs. 1-3, 5-6) gathered from the adjoint tile, completing the
//      adjoint of the particle's state after sub-step k; the reverse of G2P
//      of sub-step k added to dL/dV_k (one vector reduction per stencil node)
//      and G2P's part of the adjoint of (x, F) before it, stored by particle id;
//   3. the grid blocks it reached listed for the reverse grid operation.
// The reverse of the grid operation of sub-step k (node-local, with the tool
// frame adjoints) runs between two such launches.  A last launch applies the
// reverse of the first sub-step's P2G to the initial state.  Branches are
// held where the forward pass took them; the arithmetic is that of the
// unsorted adjoint kernels (adjoint.cuh).
#include <algorithm>

#include "adjoint.cuh"
#include "common.cuh"
#include "launch.h"

namespace gbmpm {

namespace {

constexpr int kRevThreads = 128;
// Work items are chunks of a block's particles: chunk c of block b holds its
// particles [c kChunk, (c+1) kChunk), the last of kMaxChunks the rest, so that
// the dense blocks under a tool spread over several CTAs.
constexpr uint32_t kChunk = 80, kMaxChunks = 16;

struct RevSmem {
    float4 vtile[216];      // V_k at [4b, 4b+5]^3 (.xyz)
    float4 gbt[512];        // dL/d(m, mv) of G_{k+1} at [4b-1, 4b+6]^3
    ToolFrame tools[kMaxTools];
};

// DO_G2P: reverse G2P of sub-step k (and P2G of sub-step k+1 if DO_P2G) for
// the particles recorded as sub-step k's input.  !DO_G2P: reverse P2G of the
// first sub-step at those particles themselves (v0, C0: their initial v, C).
template <bool DO_P2G, bool DO_G2P>
__global__ void __launch_bounds__(kRevThreads) k_reverse_step(DevParams P, ReverseArgs R) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RevSmem &s = *reinterpret_cast<RevSmem *>(smem_raw);
    const int tid = threadIdx.x;
    const EnvParams ep = P.envp[0];
    const int n = P.n, nb = P.nb;
    const int ntw = ep.ntools * (int)(sizeof(ToolFrame) / 4);
    if (DO_G2P)
        for (int q = tid; q < ntw; q += kRevThreads)
            reinterpret_cast<float *>(s.tools)[q] = reinterpret_cast<const float *>(R.frames)[q];
    float mub = 0.f, lamb = 0.f;
    const uint32_t nact = *R.rec.nact;
    for (uint32_t it = blockIdx.x; it < nact * kMaxChunks; it += gridDim.x) {
        const uint32_t b = R.rec.act[it % nact], chunk = it / nact;
        const uint2 brng = R.rec.blk[b];
        const uint32_t c0 = chunk * kChunk;
        if (c0 >= brng.y) continue;                  // uniform over the CTA
        const uint2 rng = make_uint2(brng.x + c0, chunk + 1 == kMaxChunks ? brng.y - c0 : min(kChunk, brng.y - c0));
        const int bx = b % nb, by = (b / nb) % nb, bz = b / (nb * nb);
        const int ox = 4 * bx, oy = 4 * by, oz = 4 * bz;
        __syncthreads();   // the previous item's tiles are consumed
        if (DO_G2P && chunk == 0 && tid < 32) {
            // list the grid blocks this block's scatter reaches, b + {0,1}^3 (lanes 0..7),
            // with one atomic on the list's count per block
            const int tx = bx + (tid & 1), ty = by + ((tid >> 1) & 1), tz = bz + ((tid >> 2) & 1);
            uint32_t tb = 0;
            bool fresh = false;
            if (tid < 8 && tx < nb && ty < nb && tz < nb) {
                tb = block_id(tx, ty, tz, nb);
                fresh = atomicExch(&R.stamp[tb], R.sv) != R.sv;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, fresh);
            uint32_t first = 0;
            if (tid == 0 && bal) first = atomicAdd(R.touch_count, (uint32_t)__popc(bal));
            first = __shfl_sync(0xffffffffu, first, 0);
            if (fresh) R.touch_list[first + __popc(bal & ((1u << tid) - 1u))] = tb;
        }
        if (DO_G2P) {
            for (int q = tid; q < 216; q += kRevThreads) {
                const int i = ox + q % 6, j = oy + (q / 6) % 6, k = oz + q / 36;
                float3 v = make_float3(0.f, 0.f, 0.f);
                if (i < n && j < n && k < n) {
                    const float4 g = R.Gk[node_addr(i, j, k, nb)];
                    v = grid_node_update(g.x, g.y, g.z, g.w, i, j, k, P, s.tools, ep.ntools);
                }
                s.vtile[q] = make_float4(v.x, v.y, v.z, 0.f);
            }
        }
        if (DO_P2G) {
            for (int q = tid; q < 512; q += kRevThreads) {
                const int i = ox - 1 + (q & 7), j = oy - 1 + ((q >> 3) & 7), k = oz - 1 + (q >> 6);
                float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i >= 0 && j >= 0 && k >= 0 && i < n && j < n && k < n) g = R.gbar_next[node_addr(i, j, k, nb)];
                s.gbt[q] = g;
            }
        }
        __syncthreads();
        // stencil nodes of a base in b, clamped to the tile as the forward G2P clamps them
        auto tile6 = [&](int b0, int b1, int b2, int ii, int jj, int kk) {
            const int lx = min(max(b0 - ox, 0), 3) + ii, ly = min(max(b1 - oy, 0), 3) + jj;
            const int lz = min(max(b2 - oz, 0), 3) + kk;
            return lx + 6 * ly + 36 * lz;
        };
        auto vel = [&](int b0, int b1, int b2, int ii, int jj, int kk) {
            const float4 g = s.vtile[tile6(b0, b1, b2, ii, jj, kk)];
            return make_float3(g.x, g.y, g.z);
        };
        // a node's velocity adjoint goes straight to dL/dV_k as one vector
        // reduction (shared float atomics into an arena were 13% slower overall)
        auto scatter = [&](int b0, int b1, int b2, int ii, int jj, int kk, float3 val) {
            const int q = tile6(b0, b1, b2, ii, jj, kk);
            const int gi = ox + q % 6, gj = oy + (q / 6) % 6, gk = oz + q / 36;
            if (gi < n && gj < n && gk < n) {
                float4 *gp = &R.vbar[node_addr(gi, gj, gk, nb)];
                asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(gp), "f"(0.f), "f"(val.x),
                             "f"(val.y), "f"(val.z)
                             : "memory");
            }
        };
        auto gtile = [&](int b0, int b1, int b2, int ii, int jj, int kk) {
            return s.gbt[(b0 - ox + 1 + ii) + 8 * (b1 - oy + 1 + jj) + 64 * (b2 - oz + 1 + kk)];
        };
        auto gglob = [&](int b0, int b1, int b2, int ii, int jj, int kk) {
            return R.gbar_next[node_addr(b0 + ii, b1 + jj, b2 + kk, nb)];
        };
        (void)gtile;
        // three lanes per particle, one z-plane of its stencils each: lanes 3g .. 3g+2
        // of a warp hold particle g of the warp's ten; rounds are warp-uniform so
        // that the lane reductions see every lane of the warp
        const int lane = tid & 31, warp = tid >> 5;
        const int grp = lane < 30 ? lane / 3 : 9, kk = lane < 30 ? lane % 3 : 0;
        const ThreeLanes red{3 * grp};
        const bool lead = lane < 30 && kk == 0;
        const uint32_t end = rng.x + rng.y;
        for (uint32_t base = rng.x + 10u * (uint32_t)warp; base < end; base += 10u * (kRevThreads / 32)) {
            const uint32_t p0 = base + (uint32_t)grp;
            const bool active = lane < 30 && p0 < end;
            const uint32_t p = active ? p0 : rng.x;          // inactive lanes compute on a valid particle
            const float4 xi = R.rec.xi[p];
            const float4 a0 = R.rec.f0[p], a1 = R.rec.f1[p];
            const float F[9] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, R.rec.f2[p]};
            const float xp[3] = {xi.x, xi.y, xi.z};
            const size_t id = __float_as_uint(xi.w);
            float xb[3], vb[3], Cb[9], Fb[9];
#pragma unroll
            for (int a = 0; a < 3; ++a) { xb[a] = R.lam.x[3 * id + a]; vb[a] = R.lam.v[3 * id + a]; }
#pragma unroll
            for (int q = 0; q < 9; ++q) { Cb[q] = R.lam.C[9 * id + q]; Fb[q] = R.lam.F[9 * id + q]; }
            // the state the reverse P2G differentiates, and where its stencil sits
            float xs[3], vs[3], Cs[9], Fs[9];
            if (DO_G2P) {
                // v and C after the sub-step as the forward pass computed them
                const float4 c0 = R.rec.vc.vc0[p], c1 = R.rec.vc.vc1[p], c2 = R.rec.vc.vc2[p];
                vs[0] = c0.x; vs[1] = c0.y; vs[2] = c0.z;
                Cs[0] = c0.w; Cs[1] = c1.x; Cs[2] = c1.y; Cs[3] = c1.z; Cs[4] = c1.w;
                Cs[5] = c2.x; Cs[6] = c2.y; Cs[7] = c2.z; Cs[8] = c2.w;
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        Fs[3 * r + c] = F[3 * r + c] + P.dt * (Cs[3 * r] * F[c] + Cs[3 * r + 1] * F[3 + c] +
                                                               Cs[3 * r + 2] * F[6 + c]);
#pragma unroll
                for (int a = 0; a < 3; ++a) xs[a] = xp[a] + P.dt * vs[a];
            } else {
#pragma unroll
                for (int a = 0; a < 3; ++a) { xs[a] = xp[a]; vs[a] = R.v0[3 * id + a]; }
#pragma unroll
                for (int q = 0; q < 9; ++q) { Cs[q] = R.C0[9 * id + q]; Fs[q] = F[q]; }
            }
            if (DO_P2G) {
                uint32_t err = 0;
                int hb[3];
                stencil_axis(xs[0], P.inv_dx, n, hb[0], err);
                stencil_axis(xs[1], P.inv_dx, n, hb[1], err);
                stencil_axis(xs[2], P.inv_dx, n, hb[2], err);
                const bool in_tile = hb[0] - ox >= -1 && hb[0] - ox <= 4 && hb[1] - oy >= -1 && hb[1] - oy <= 4 &&
                                     hb[2] - oz >= -1 && hb[2] - oz <= 4;
                float vbn[3], Cbn[9];
                if (__all_sync(0xffffffffu, in_tile))
                    adj_p2g_particle(P, ep, xs, vs, Cs, Fs, gtile, xb, Fb, vbn, Cbn, mub, lamb, kk, 1, red,
                                     lead && active);
                else
                    adj_p2g_particle(P, ep, xs, vs, Cs, Fs, gglob, xb, Fb, vbn, Cbn, mub, lamb, kk, 1, red,
                                     lead && active);
#pragma unroll
                for (int a = 0; a < 3; ++a) vb[a] += vbn[a];
#pragma unroll
                for (int q = 0; q < 9; ++q) Cb[q] += Cbn[q];
            }
            if (DO_G2P) {
                float xbn[3], Fbn[9];
                auto scatter_if = [&](int b0, int b1, int b2, int ii, int jj, int kq, float3 val) {
                    if (active) scatter(b0, b1, b2, ii, jj, kq, val);
                };
                adj_g2p_particle(P, xp, F, vel, xb, vb, Cb, Fb, scatter_if, xbn, Fbn, kk, 1, red, Cs);
                if (lead && active) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) { R.lam.x[3 * id + a] = xbn[a]; R.lam.v[3 * id + a] = 0.f; }
#pragma unroll
                    for (int q = 0; q < 9; ++q) { R.lam.F[9 * id + q] = Fbn[q]; R.lam.C[9 * id + q] = 0.f; }
                }
            } else if (lead && active) {
#pragma unroll
                for (int a = 0; a < 3; ++a) { R.lam.x[3 * id + a] = xb[a]; R.lam.v[3 * id + a] = vb[a]; }
#pragma unroll
                for (int q = 0; q < 9; ++q) { R.lam.F[9 * id + q] = Fb[q]; R.lam.C[9 * id + q] = Cb[q]; }
            }
        }
    }
    if (DO_P2G) {
        // the CTA's part of dL/dmu, dL/dlambda, added to its own pair of the
        // per-CTA partial sums (no two CTAs share a pair, so no atomics)
        __shared__ double red_s[2][kRevThreads / 32];
        mub = warp_sum(mub);
        lamb = warp_sum(lamb);
        __syncthreads();
        if ((tid & 31) == 0) { red_s[0][tid >> 5] = mub; red_s[1][tid >> 5] = lamb; }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, c = 0.0;
            for (int w = 0; w < kRevThreads / 32; ++w) { a += red_s[0][w]; c += red_s[1][w]; }
            R.lame_part[2 * blockIdx.x] += a;
            R.lame_part[2 * blockIdx.x + 1] += c;
        }
    }
}

template <bool DO_P2G, bool DO_G2P>
int reverse_occupancy() {
    constexpr int bytes = (int)sizeof(RevSmem);
    cudaFuncSetAttribute(k_reverse_step<DO_P2G, DO_G2P>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_reverse_step<DO_P2G, DO_G2P>, kRevThreads, bytes);
    return a;
}

}  // namespace

int reverse_step_ctas_per_sm() {
    const int a = reverse_occupancy<true, true>(), b = reverse_occupancy<false, true>(),
              c = reverse_occupancy<true, false>();
    return std::min(a, std::min(b, c));
}

void launch_reverse_step(bool do_p2g, bool do_g2p, const DevParams &P, const ReverseArgs &R, int grid,
                         cudaStream_t st) {
    const size_t bytes = sizeof(RevSmem);
    if (do_p2g && do_g2p)
        k_reverse_step<true, true><<<grid, kRevThreads, bytes, st>>>(P, R);
    else if (do_g2p)
        k_reverse_step<false, true><<<grid, kRevThreads, bytes, st>>>(P, R);
    else if (do_p2g)
        k_reverse_step<true, false><<<grid, kRevThreads, bytes, st>>>(P, R);
}

}  // namespace gbmpm
