// kernels_adjoint.cu -- reverse mode of one sub-step of the split pipeline
// (particles in load order, one blocked n^3 grid), for gradients of a loss of
// the state after a rollout with respect to the material (mu, lambda of
// Eq. 6), the tool frames of every sub-step (and through them the tool
// poses) and the initial state.
//
// Each sub-step is differentiated stage by stage in reverse order: G2P
// (Eqs. 4, 8-10), the grid operation (Eq. 7, gravity, Eqs. 11-19, walls) and
// P2G (Eqs. 1-3 with the stress of Eqs. 5-6).  Every branch the forward pass
// takes (m > 0, walls, contact d < theta, approaching v_n < 0, the friction
// clamp, the closest tool) is held fixed; distances only select branches;
// sampled fields are piecewise constant in x_ref and have no normal
// derivative.
#include "adjoint.cuh"
#include "common.cuh"
#include "launch.h"

namespace gbmpm {

namespace {

constexpr int kThreads = 256;

// --------------------------------------------------------------- G2P

// From the adjoint of (x', v', C', F') of each particle to the adjoint of the
// grid velocities (scattered into Gb.yzw) and G2P's part of the adjoint of
// (x, F); v and C do not enter G2P, so their adjoints are cleared here.
__global__ void __launch_bounds__(kThreads) k_adj_g2p(DevParams P, PState S, uint32_t n,
                                                       const float4 *__restrict__ Gv, AdjState A,
                                                       float4 *__restrict__ Gb, VCState Vn) {
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const float4 xi = S.xi[s];
        const float xp[3] = {xi.x, xi.y, xi.z};
        const float4 a0 = S.f0[s], a1 = S.f1[s];
        const float F[9] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, S.f2[s]};
        float xbo[3], vbo[3], Cbo[9], Fbo[9];
#pragma unroll
        for (int a = 0; a < 3; ++a) { xbo[a] = A.x[3 * (size_t)s + a]; vbo[a] = A.v[3 * (size_t)s + a]; }
#pragma unroll
        for (int q = 0; q < 9; ++q) { Cbo[q] = A.C[9 * (size_t)s + q]; Fbo[q] = A.F[9 * (size_t)s + q]; }
        const int nb = P.nb;
        auto vel = [&](int bx, int by, int bz, int ii, int jj, int kk) {
            const float4 g = Gv[node_addr(bx + ii, by + jj, bz + kk, nb)];
            return make_float3(g.y, g.z, g.w);
        };
        auto scatter = [&](int bx, int by, int bz, int ii, int jj, int kk, float3 v) {
            atomicAdd(&Gb[node_addr(bx + ii, by + jj, bz + kk, nb)], make_float4(0.f, v.x, v.y, v.z));
        };
        float xbn[3], Fbn[9];
        if (Vn.vc0) {
            // v and C after the sub-step, as the forward pass wrote them
            const float4 c0 = Vn.vc0[s], c1 = Vn.vc1[s], c2 = Vn.vc2[s];
            const float vnew[3] = {c0.x, c0.y, c0.z};
            const float Cnew[9] = {c0.w, c1.x, c1.y, c1.z, c1.w, c2.x, c2.y, c2.z, c2.w};
            adj_g2p_particle<decltype(vel), decltype(scatter), OneLane, true>(P, xp, F, vel, xbo, vbo, Cbo, Fbo,
                                                                              scatter, xbn, Fbn, 0, 3, OneLane(),
                                                                              Cnew, vnew);
        } else {
            adj_g2p_particle<decltype(vel), decltype(scatter), OneLane, true>(P, xp, F, vel, xbo, vbo, Cbo, Fbo,
                                                                              scatter, xbn, Fbn);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) { A.x[3 * (size_t)s + a] = xbn[a]; A.v[3 * (size_t)s + a] = 0.f; }
#pragma unroll
        for (int q = 0; q < 9; ++q) { A.F[9 * (size_t)s + q] = Fbn[q]; A.C[9 * (size_t)s + q] = 0.f; }
    }
}

// ------------------------------------------------------ grid operation

// The reverse grid operation at node g (grid (m, mv) node, incoming velocity
// adjoint gb.yzw), with the tool-frame adjoints summed over the warp.  Called
// by all 32 lanes of a warp together.
__device__ __forceinline__ void adj_grid_node(const DevParams &P, const ToolFrame *s_tools, int ntools,
                                              float4 *__restrict__ Gb, double *__restrict__ tool_bar, uint32_t g,
                                              float4 node, float4 gb, int lo, int hi) {
    const uint32_t blk = g >> 6, l = g & 63u;
    const int bx = blk % P.nb, by = (blk / P.nb) % P.nb, bz = blk / (P.nb * P.nb);
    const int i = bx * 4 + (l & 3), j = by * 4 + ((l >> 2) & 3), k = bz * 4 + (l >> 4);
    float tb[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) tb[q] = 0.f;
    int hit = -1;
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    const bool wall = i < lo || j < lo || k < lo || i >= hi || j >= hi || k >= hi;
    if (node.x > 0.0f && !wall) {
        const float m = node.x;
        const float vf[3] = {node.y / m + P.dt * P.gx, node.z / m + P.dt * P.gy, node.w / m + P.dt * P.gz};
        float vbar[3] = {gb.y, gb.z, gb.w};
        if (ntools > 0) {
            const float xw[3] = {i * P.dx, j * P.dx, k * P.dx};
            float dmin, nr[3], pr[3];
            const int id = nearest_tool(xw[0], xw[1], xw[2], s_tools, ntools, dmin, nr[0], nr[1], nr[2], pr[0],
                                        pr[1], pr[2]);
            if (id >= 0 && dmin < P.theta) {
                const ToolFrame &tf = s_tools[id];
                float nw[3], r[3], vco[3], vrel[3], vn = 0.f;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    nw[a] = tf.R[3 * a] * nr[0] + tf.R[3 * a + 1] * nr[1] + tf.R[3 * a + 2] * nr[2];
                    r[a] = xw[a] - tf.T[a];
                }
                vco[0] = tf.u[0] + tf.w[1] * r[2] - tf.w[2] * r[1];
                vco[1] = tf.u[1] + tf.w[2] * r[0] - tf.w[0] * r[2];
                vco[2] = tf.u[2] + tf.w[0] * r[1] - tf.w[1] * r[0];
#pragma unroll
                for (int a = 0; a < 3; ++a) { vrel[a] = vf[a] - vco[a]; vn += vrel[a] * nw[a]; }   // Eqs. 15-16
                if (vn < 0.0f) {
                    hit = id;
                    float vt[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) vt[a] = vrel[a] - vn * nw[a];                      // Eq. 17
                    const float tn = sqrtf(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]);
                    float scale = 0.f;
                    if (tn > 0.0f) scale = fmaxf(tn + P.fric * vn, 0.0f) / tn;                   // Eq. 18
                    // v' = scale vt + vco (Eq. 19)
                    float vtb[3] = {0.f, 0.f, 0.f}, vnb = 0.f;
                    if (scale > 0.f) {
                        const float scb = vbar[0] * vt[0] + vbar[1] * vt[1] + vbar[2] * vt[2];
                        vnb += P.fric * scb / tn;                 // scale = 1 + mu_f vn / |vt|
                        const float vtnb = -P.fric * vn * scb / (tn * tn);
#pragma unroll
                        for (int a = 0; a < 3; ++a) vtb[a] = scale * vbar[a] + vtnb * vt[a] / tn;
                    }
                    float vrelb[3], nwb[3];
                    const float vtb_n = vtb[0] * nw[0] + vtb[1] * nw[1] + vtb[2] * nw[2];
                    vnb -= vtb_n;                                 // vt = vrel - vn nw
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        vrelb[a] = vtb[a] + vnb * nw[a];          // vn = vrel . nw
                        nwb[a] = -vn * vtb[a] + vnb * vrel[a];
                    }
                    float vcob[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) vcob[a] = vbar[a] - vrelb[a];   // vrel = v - vco; v' has + vco
                    // vco = u + w x r, r = x - T
#pragma unroll
                    for (int a = 0; a < 3; ++a) tb[12 + a] = vcob[a];
                    tb[15] = r[1] * vcob[2] - r[2] * vcob[1];
                    tb[16] = r[2] * vcob[0] - r[0] * vcob[2];
                    tb[17] = r[0] * vcob[1] - r[1] * vcob[0];
                    tb[9] = -(vcob[1] * tf.w[2] - vcob[2] * tf.w[1]);
                    tb[10] = -(vcob[2] * tf.w[0] - vcob[0] * tf.w[2]);
                    tb[11] = -(vcob[0] * tf.w[1] - vcob[1] * tf.w[0]);
                    // nw = R n_ref(x_ref), x_ref = R^T (x - T)
                    float nrb[3], Jn[9], xrb[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int c = 0; c < 3; ++c) tb[3 * a + c] = nwb[a] * nr[c];
#pragma unroll
                    for (int c = 0; c < 3; ++c) nrb[c] = tf.R[c] * nwb[0] + tf.R[3 + c] * nwb[1] + tf.R[6 + c] * nwb[2];
                    tool_normal_jacobian(tf.kind, tf.dims, pr[0], pr[1], pr[2], Jn);
#pragma unroll
                    for (int c = 0; c < 3; ++c) xrb[c] = Jn[c] * nrb[0] + Jn[3 + c] * nrb[1] + Jn[6 + c] * nrb[2];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
#pragma unroll
                        for (int a = 0; a < 3; ++a) tb[3 * c + a] += r[c] * xrb[a];
                        tb[9 + c] -= tf.R[3 * c] * xrb[0] + tf.R[3 * c + 1] * xrb[1] + tf.R[3 * c + 2] * xrb[2];
                    }
#pragma unroll
                    for (int a = 0; a < 3; ++a) vbar[a] = vrelb[a];
                }
            }
        }
        // v = mv / m + dt g
        out = make_float4(-(vbar[0] * node.y + vbar[1] * node.z + vbar[2] * node.w) / (m * m), vbar[0] / m,
                          vbar[1] / m, vbar[2] / m);
    }
    Gb[g] = out;
    for (int t = 0; t < ntools; ++t) {
        const bool mine = hit == t;
        if (!__any_sync(0xffffffffu, mine)) continue;
#pragma unroll
        for (int q = 0; q < 18; ++q) {
            const float v = warp_sum(mine ? tb[q] : 0.f);
            if ((threadIdx.x & 31) == 0) atomicAdd(&tool_bar[18 * t + q], (double)v);
        }
    }
}

// Gb.yzw holds dL/d(grid velocity) on entry; on return Gb = (dL/dm, dL/dmv).
// G holds the grid (m, mv) the forward grid operation read.  tool_bar
// (ntools x 18: R row-major, T, u, w) accumulates dL/d(frame entries).
// L.list (if not NULL): only the nodes of those grid blocks (the others hold
// no adjoint), 8 entries per work-list block, kNoBlock entries skipped.
// L.zlist: the nodes of those blocks are cleared in L.zbuf.
__global__ void __launch_bounds__(kThreads, 3) k_adj_grid(DevParams P, const float4 *__restrict__ G,
                                                        const ToolFrame *__restrict__ tools,
                                                        float4 *__restrict__ Gb, double *__restrict__ tool_bar,
                                                        AdjGridLists L) {
    // the next reverse sub-step's record was written a segment's replay ago and
    // has left L2: start bringing it back (independent of the previous launch)
    if (L.prefetch) {
        const char *pf = static_cast<const char *>(L.prefetch);
        for (size_t off = (size_t)(blockIdx.x * blockDim.x + threadIdx.x) * 128u; off < L.prefetch_bytes;
             off += (size_t)gridDim.x * blockDim.x * 128u)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(pf + off));
    }
    // a programmatic dependent of the reverse sub-step: its results are read
    // after the wait; the next reverse sub-step is released after it too
    griddep_wait();
    griddep_launch_dependents();
    const int ntools = P.envp[0].ntools;
    const int lo = P.bound, hi = P.n - P.bound;
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    if (!L.list) {
        // every node (n^3 is a multiple of 64, so whole warps stay in the loop), the
        // tool frames from a shared copy
        __shared__ ToolFrame s_tools[kMaxTools];
        if (threadIdx.x < ntools * (sizeof(ToolFrame) / 4))
            reinterpret_cast<float *>(s_tools)[threadIdx.x] = reinterpret_cast<const float *>(tools)[threadIdx.x];
        __syncthreads();
        const uint32_t total = (uint32_t)P.n * P.n * P.n;
        for (uint32_t q = gt; q < total; q += stride)
            adj_grid_node(P, s_tools, ntools, Gb, tool_bar, q, G[q], Gb[q], lo, hi);
        return;
    }
    // the listed blocks: the tool frames are read through L1 (no shared copy, so
    // no barrier before the first node)
    // one thread per node of the listed blocks (the 64 threads of an entry read
    // the same entry, so an empty one is skipped by whole warps)
    const uint32_t total = *L.nlist * 512u, zt = L.zlist ? *L.znlist * 512u : 0u;
    for (uint32_t q = gt; q < max(total, zt); q += stride) {
        const uint32_t zb = q < zt ? L.zlist[q >> 6] : kNoBlock, tb = q < total ? L.list[q >> 6] : kNoBlock;
        if (zb != kNoBlock) L.zbuf[zb * 64u + (q & 63u)] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (tb == kNoBlock) continue;
        const uint32_t g = tb * 64u + (q & 63u);
        adj_grid_node(P, tools, ntools, Gb, tool_bar, g, G[g], Gb[g], lo, hi);
    }
}

// ---------------------------------------------------------------- P2G

// From Gb = (dL/dm, dL/dmv) to the adjoint of (x, v, C, F): adds to G2P's
// parts in A.x and A.F, writes A.v and A.C; lame_bar[2] accumulates
// dL/dmu, dL/dlambda.
__global__ void __launch_bounds__(kThreads) k_adj_p2g(DevParams P, PState S, VCState V, uint32_t n,
                                                       const float4 *__restrict__ Gb, AdjState A,
                                                       double *__restrict__ lame_bar) {
    const EnvParams ep = P.envp[0];
    float mub = 0.f, lamb = 0.f;
    const uint32_t span = (n + 31u) & ~31u;            // whole warps for the reduction
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < span; s += gridDim.x * blockDim.x) {
        if (s < n) {
            const float4 xi = S.xi[s];
            const float xp[3] = {xi.x, xi.y, xi.z};
            const float4 a0 = S.f0[s], a1 = S.f1[s];
            const float F[9] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, S.f2[s]};
            const float4 c0 = V.vc0[s], c1 = V.vc1[s], c2 = V.vc2[s];
            const float vp[3] = {c0.x, c0.y, c0.z};
            const float C[9] = {c0.w, c1.x, c1.y, c1.z, c1.w, c2.x, c2.y, c2.z, c2.w};
            const int nb = P.nb;
            auto gbar = [&](int bx, int by, int bz, int ii, int jj, int kk) {
                return Gb[node_addr(bx + ii, by + jj, bz + kk, nb)];
            };
            float xb[3], Fb[9], vb[3], Cb[9];
#pragma unroll
            for (int a = 0; a < 3; ++a) xb[a] = A.x[3 * (size_t)s + a];
#pragma unroll
            for (int q = 0; q < 9; ++q) Fb[q] = A.F[9 * (size_t)s + q];
            adj_p2g_particle<decltype(gbar), OneLane, true>(P, ep, xp, vp, C, F, gbar, xb, Fb, vb, Cb, mub, lamb);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                A.x[3 * (size_t)s + a] = xb[a];
                A.v[3 * (size_t)s + a] = vb[a];
            }
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                A.F[9 * (size_t)s + q] = Fb[q];
                A.C[9 * (size_t)s + q] = Cb[q];
            }
        }
    }
    mub = warp_sum(mub);
    lamb = warp_sum(lamb);
    if ((threadIdx.x & 31) == 0 && (mub != 0.f || lamb != 0.f)) {
        atomicAdd(&lame_bar[0], (double)mub);
        atomicAdd(&lame_bar[1], (double)lamb);
    }
}

}  // namespace

void launch_adj_g2p(const DevParams &P, const PState &S, uint32_t n, const float4 *Gv, const AdjState &A, float4 *Gb,
                    const VCState &Vnext, int grid, cudaStream_t st) {
    if (n == 0) return;
    k_adj_g2p<<<grid, kThreads, 0, st>>>(P, S, n, Gv, A, Gb, Vnext);
}
void launch_adj_grid(const DevParams &P, const float4 *G, const ToolFrame *tools, float4 *Gb, double *tool_bar,
                     int grid, cudaStream_t st, const AdjGridLists &L) {
    if (L.list)   // the fused reverse pass: a programmatic dependent of the reverse sub-step
        launch_dependent(k_adj_grid, grid, kThreads, 0, st, P, G, tools, Gb, tool_bar, L);
    else
        k_adj_grid<<<grid, kThreads, 0, st>>>(P, G, tools, Gb, tool_bar, L);
}
void launch_adj_p2g(const DevParams &P, const PState &S, const VCState &V, uint32_t n, const float4 *Gb,
                    const AdjState &A, double *lame_bar, int grid, cudaStream_t st) {
    if (n == 0) return;
    k_adj_p2g<<<grid, kThreads, 0, st>>>(P, S, V, n, Gb, A, lame_bar);
}

}  // namespace gbmpm
