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
#include <type_traits>

#include "adjoint.cuh"
#include "common.cuh"
#include "launch.h"

namespace gbmpm {

namespace {

constexpr int kRevThreads = 128;
// Work items are chunks of a block's particles: chunk c of block b holds its
// particles [c kChunk, (c+1) kChunk), the last of kMaxChunks the rest, so that
// the dense blocks under a tool spread over several CTAs.
constexpr uint32_t kChunk = 128, kMaxChunks = 16;
// Lanes per particle: 1 (the whole stencil; a chunk is then one round of the
// CTA) or 3 (one z-plane of the stencil each, partials summed by shuffles),
// which made the whole backward 4% slower.
constexpr int kRevLanes = 1;

struct RevSmem {
    float4 vtile[216];      // V_k at [4b, 4b+5]^3 (.xyz)
    float4 gbt[512];        // dL/d(m, mv) of G_{k+1} at [4b-1, 4b+6]^3
};

// One particle's recorded inputs of a reverse sub-step: state before the
// sub-step (xi = x | id, F), v and C after it, and the incoming (x, F) adjoint
// by position
struct RevIn {
    float4 xi, a0, a1, c0, c1, c2, l0, l1, l2;
    float f2;
};
// the recorded part (written by the replay, before the previous reverse launch)
template <bool DO_G2P>
__device__ __forceinline__ void load_rev_rec(const ReverseArgs &R, uint32_t p, RevIn &in) {
    in.xi = R.rec.xi[p];
    in.a0 = R.rec.f0[p];
    in.a1 = R.rec.f1[p];
    in.f2 = R.rec.f2[p];
    if (DO_G2P) {
        in.c0 = R.rec.vc.vc0[p];
        in.c1 = R.rec.vc.vc1[p];
        in.c2 = R.rec.vc.vc2[p];
    }
}
// the incoming adjoint by position (written by the previous reverse launch)
template <bool DO_G2P>
__device__ __forceinline__ void load_rev_lam(const ReverseArgs &R, uint32_t p, RevIn &in) {
    if (DO_G2P && !R.lam_in_by_id) {
        in.l0 = R.lp_in[p];
        in.l1 = R.lp_in[R.np + p];
        in.l2 = R.lp_in[2 * R.np + p];
    }
}

// DO_G2P: reverse G2P of sub-step k (and P2G of sub-step k+1 if DO_P2G) for
// the particles recorded as sub-step k's input.  !DO_G2P: reverse P2G of the
// first sub-step at those particles themselves (v0, C0: their initial v, C).
template <bool DO_P2G, bool DO_G2P, int LANES = kRevLanes>
__global__ void __launch_bounds__(kRevThreads) k_reverse_step(DevParams P, ReverseArgs R) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RevSmem &s = *reinterpret_cast<RevSmem *>(smem_raw);
    const int tid = threadIdx.x;
    const EnvParams ep = P.envp[0];
    const int n = P.n, nb = P.nb;
    float mub = 0.f, lamb = 0.f;
    // Launched as a programmatic dependent of the previous launch: until
    // griddep_wait() only the record is read (and this sub-step's own list
    // slot written), so the first item's set-up overlaps the previous launch.
    // The next launch is released only after the wait, so it overlaps this one
    // alone (whose list slots and buffers it does not touch before its wait).
    bool waited = false;
    const uint32_t nact = *R.rec.nact;
    if (DO_G2P && blockIdx.x == 0 && tid == 0) *R.touch_n = nact;
    for (uint32_t it = blockIdx.x; it < nact * kMaxChunks; it += gridDim.x) {
        const uint32_t ai = it % nact, chunk = it / nact;
        const uint32_t b = R.rec.act[ai];
        const uint2 brng = R.rec.blk[ai];
        const uint32_t c0 = chunk * kChunk;
        if (c0 >= brng.y) {                          // uniform over the CTA
            if (DO_G2P && chunk == 0 && tid < 8) R.touch_list[8 * it + tid] = kNoBlock;
            continue;
        }
        const uint2 rng = make_uint2(brng.x + c0, chunk + 1 == kMaxChunks ? brng.y - c0 : min(kChunk, brng.y - c0));
        const int bx = b % nb, by = (b / nb) % nb, bz = b / (nb * nb);
        const int ox = 4 * bx, oy = 4 * by, oz = 4 * bz;
        // LANES == 3: lanes 3g .. 3g+2 of a warp hold particle g of the warp's ten, one
        // z-plane of its stencils each; rounds are warp-uniform so that the lane
        // reductions see every lane of the warp.  LANES == 1: one particle per lane.
        const int lane = tid & 31, warp = tid >> 5;
        constexpr uint32_t kPerWarp = LANES == 3 ? 10u : 32u;
        const int grp = LANES == 3 ? (lane < 30 ? lane / 3 : 9) : lane;
        const uint32_t end = rng.x + rng.y;
        // the first round's inputs, loaded now so that they arrive during the tiles
        const uint32_t base0 = rng.x + kPerWarp * (uint32_t)warp;
        const uint32_t pin0 = base0 + (uint32_t)grp < end ? base0 + (uint32_t)grp : rng.x;
        RevIn in0;
        load_rev_rec<DO_G2P>(R, pin0, in0);
        __syncthreads();   // the previous item's tiles are consumed
        if (DO_G2P) {
            // the grid velocities of sub-step k as its grid operation left them
            for (int q = tid; q < 216; q += kRevThreads) {
                const int i = ox + q % 6, j = oy + (q / 6) % 6, k = oz + q / 36;
                s.vtile[q] = (i < n && j < n && k < n) ? R.rec.vgrid[node_addr(i, j, k, nb)]
                                                        : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        if (!waited) {
            griddep_wait();      // the previous launches' results are complete and visible
            griddep_launch_dependents();
            waited = true;
        }
        load_rev_lam<DO_G2P>(R, pin0, in0);
        // the grid blocks this block's scatter reaches, b + {0,1}^3: threads 0..7 claim
        // them through the stamps (issued here, the result used at the end of the item)
        // and fill the block's 8 entries of the touched list (it is b's index in the list)
        const bool marks = DO_G2P && chunk == 0 && tid < 8;
        uint32_t tb = kNoBlock, old = R.sv;
        if (marks) {
            const int tx = bx + (tid & 1), ty = by + ((tid >> 1) & 1), tz = bz + ((tid >> 2) & 1);
            if (tx < nb && ty < nb && tz < nb) {
                tb = block_id(tx, ty, tz, nb);
                old = atomicExch(&R.stamp[tb], R.sv);
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
        auto gtile = [&](int b0, int b1, int b2, int ii, int jj, int kk) {
            return s.gbt[(b0 - ox + 1 + ii) + 8 * (b1 - oy + 1 + jj) + 64 * (b2 - oz + 1 + kk)];
        };
        auto gglob = [&](int b0, int b1, int b2, int ii, int jj, int kk) {
            return R.gbar_next[node_addr(b0 + ii, b1 + jj, b2 + kk, nb)];
        };
        (void)gtile;
        const int kk = LANES == 3 ? (lane < 30 ? lane % 3 : 0) : 0;
        constexpr int nkk = LANES == 3 ? 1 : 3;
        using Red = typename std::conditional<LANES == 3, ThreeLanes, OneLane>::type;
        Red red;
        if constexpr (LANES == 3) red.l0 = 3 * grp;
        const bool lead = LANES == 3 ? (lane < 30 && kk == 0) : true;
        for (uint32_t base = base0; base < end; base += kPerWarp * (kRevThreads / 32)) {
            const uint32_t p0 = base + (uint32_t)grp;
            const bool active = (LANES == 1 || lane < 30) && p0 < end;
            const uint32_t p = active ? p0 : rng.x;          // inactive lanes compute on a valid particle
            RevIn in;
            if (base == base0) {
                in = in0;
            } else {
                load_rev_rec<DO_G2P>(R, p, in);
                load_rev_lam<DO_G2P>(R, p, in);
            }
            const float4 xi = in.xi, a0 = in.a0, a1 = in.a1;
            const float F[9] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, in.f2};
            const float xp[3] = {xi.x, xi.y, xi.z};
            const size_t id = min(__float_as_uint(xi.w), R.np - 1u);   // clamped: a record is never read out of range
            float xb[3], vb[3], Cb[9], Fb[9];
            if (!DO_G2P || R.lam_in_by_id) {
#pragma unroll
                for (int a = 0; a < 3; ++a) { xb[a] = R.lam.x[3 * id + a]; vb[a] = R.lam.v[3 * id + a]; }
#pragma unroll
                for (int q = 0; q < 9; ++q) { Cb[q] = R.lam.C[9 * id + q]; Fb[q] = R.lam.F[9 * id + q]; }
            } else {
                const float4 l0 = in.l0, l1 = in.l1, l2 = in.l2;
                xb[0] = l0.x; xb[1] = l0.y; xb[2] = l0.z;
                Fb[0] = l0.w; Fb[1] = l1.x; Fb[2] = l1.y; Fb[3] = l1.z; Fb[4] = l1.w;
                Fb[5] = l2.x; Fb[6] = l2.y; Fb[7] = l2.z; Fb[8] = l2.w;
#pragma unroll
                for (int a = 0; a < 3; ++a) vb[a] = 0.f;
#pragma unroll
                for (int q = 0; q < 9; ++q) Cb[q] = 0.f;
            }
            // the state the reverse P2G differentiates, and where its stencil sits
            float xs[3], vs[3], Cs[9], Fs[9];
            if (DO_G2P) {
                // v and C after the sub-step as the forward pass computed them
                const float4 c0 = in.c0, c1 = in.c1, c2 = in.c2;
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
                    adj_p2g_particle(P, ep, xs, vs, Cs, Fs, gtile, xb, Fb, vbn, Cbn, mub, lamb, kk, nkk, red,
                                     lead && active);
                else
                    adj_p2g_particle(P, ep, xs, vs, Cs, Fs, gglob, xb, Fb, vbn, Cbn, mub, lamb, kk, nkk, red,
                                     lead && active);
#pragma unroll
                for (int a = 0; a < 3; ++a) vb[a] += vbn[a];
#pragma unroll
                for (int q = 0; q < 9; ++q) Cb[q] += Cbn[q];
            }
            if (DO_G2P) {
                // node (i, j, k) sits at node_addr = ax(i) + ay(j) + az(k): the three parts
                // of this particle's (clamped) stencil nodes, and which lie in the grid
                uint32_t axo[3], ayo[3], azo[3], okm = 0u;
                {
                    uint32_t e2 = 0;
                    int hb[3];
                    stencil_axis(xp[0], P.inv_dx, n, hb[0], e2);
                    stencil_axis(xp[1], P.inv_dx, n, hb[1], e2);
                    stencil_axis(xp[2], P.inv_dx, n, hb[2], e2);
                    const int gx = ox + min(max(hb[0] - ox, 0), 3), gy = oy + min(max(hb[1] - oy, 0), 3);
                    const int gz = oz + min(max(hb[2] - oz, 0), 3);
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const uint32_t x = (uint32_t)(gx + i), y = (uint32_t)(gy + i), z = (uint32_t)(gz + i);
                        axo[i] = 64u * (x >> 2) + (x & 3u);
                        ayo[i] = 64u * (uint32_t)nb * (y >> 2) + 4u * (y & 3u);
                        azo[i] = 64u * (uint32_t)nb * (uint32_t)nb * (z >> 2) + 16u * (z & 3u);
                        okm |= ((x < (uint32_t)n) ? 1u : 0u) << i;
                        okm |= ((y < (uint32_t)n) ? 1u : 0u) << (3 + i);
                        okm |= ((z < (uint32_t)n) ? 1u : 0u) << (6 + i);
                    }
                    if (!active) okm = 0u;
                }
                // a node's velocity adjoint goes straight to dL/dV_k as one vector
                // reduction (shared float atomics into an arena were 13% slower overall)
                auto scatter = [&](int, int, int, int ii, int jj, int kq, float3 val) {
                    if ((okm >> ii) & (okm >> (3 + jj)) & (okm >> (6 + kq)) & 1u) {
                        float4 *gp = &R.vbar[axo[ii] + ayo[jj] + pick3(azo, kq)];
                        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(gp), "f"(0.f), "f"(val.x),
                                     "f"(val.y), "f"(val.z)
                                     : "memory");
                    }
                };
                float xbn[3], Fbn[9];
                adj_g2p_particle(P, xp, F, vel, xb, vb, Cb, Fb, scatter, xbn, Fbn, kk, nkk, red, Cs, vs);
                if (lead && active) {
                    if (R.lam_out_by_id) {
#pragma unroll
                        for (int a = 0; a < 3; ++a) { R.lam.x[3 * id + a] = xbn[a]; R.lam.v[3 * id + a] = 0.f; }
#pragma unroll
                        for (int q = 0; q < 9; ++q) { R.lam.F[9 * id + q] = Fbn[q]; R.lam.C[9 * id + q] = 0.f; }
                    } else {
                        const uint32_t q = min(R.rec.src[p], R.np - 1u);
                        R.lp_out[q] = make_float4(xbn[0], xbn[1], xbn[2], Fbn[0]);
                        R.lp_out[R.np + q] = make_float4(Fbn[1], Fbn[2], Fbn[3], Fbn[4]);
                        R.lp_out[2 * R.np + q] = make_float4(Fbn[5], Fbn[6], Fbn[7], Fbn[8]);
                    }
                }
            } else if (lead && active) {
#pragma unroll
                for (int a = 0; a < 3; ++a) { R.lam.x[3 * id + a] = xb[a]; R.lam.v[3 * id + a] = vb[a]; }
#pragma unroll
                for (int q = 0; q < 9; ++q) { R.lam.F[9 * id + q] = Fb[q]; R.lam.C[9 * id + q] = Cb[q]; }
            }
        }
        // the claimed blocks, stored last: the stamp exchanges ran during the item
        if (marks) R.touch_list[8 * it + tid] = old != R.sv ? tb : kNoBlock;
    }
    if (!waited) griddep_wait();     // a CTA without particles still adds to its pair below
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
                         cudaStream_t st, bool dependent) {
    const size_t bytes = sizeof(RevSmem);
    auto go = [&](auto kernel) {
        if (dependent)
            launch_dependent(kernel, grid, kRevThreads, bytes, st, P, R);
        else
            kernel<<<grid, kRevThreads, bytes, st>>>(P, R);
    };
    if (do_p2g && do_g2p)
        go(k_reverse_step<true, true>);
    else if (do_g2p)
        go(k_reverse_step<false, true>);
    else if (do_p2g)
        go(k_reverse_step<true, false>);
}

}  // namespace gbmpm
