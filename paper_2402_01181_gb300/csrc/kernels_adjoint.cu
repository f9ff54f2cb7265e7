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
#include "common.cuh"
#include "launch.h"

namespace gbmpm {

namespace {

constexpr int kThreads = 256;

// d w / d fx of bspline_weights
__device__ __forceinline__ void bspline_slopes(float fx, float d[3]) {
    d[0] = fx - 1.5f;
    d[1] = -2.0f * (fx - 1.0f);
    d[2] = fx - 0.5f;
}

// Jacobian d n_ref / d p_ref (row = component of n) of tool_sdf's unit normal;
// zero where that normal is constant (inside a box, on a capsule's axis).
__device__ __forceinline__ void tool_normal_jacobian(int kind, const float *dims, float px, float py, float pz,
                                                     float J[9]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) J[q] = 0.f;
    if (kind == 0) {
        const float c = fminf(fmaxf(py, -dims[1]), dims[1]);
        const float dy = (c == py) ? 0.f : 1.f;    // d q_y / d p_y: 0 along the side, 1 on the caps
        const float q[3] = {px, py - c, pz};
        const float L2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
        if (!(L2 > 0.f)) return;
        const float iL = 1.0f / sqrtf(L2);
        const float u[3] = {q[0] * iL, q[1] * iL, q[2] * iL};
        const float D[3] = {1.f, dy, 1.f};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) J[3 * a + b] = ((a == b ? 1.f : 0.f) - u[a] * u[b]) * iL * D[b];
        return;
    }
    if (kind == 1) {
        const float p[3] = {px, py, pz};
        float o[3], s[3], o2 = 0.f;
        bool act[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float q = fabsf(p[d]) - dims[d];
            act[d] = q > 0.f;
            o[d] = fmaxf(q, 0.f);
            s[d] = p[d] < 0.f ? -1.f : 1.f;
            o2 += o[d] * o[d];
        }
        if (!(o2 > 0.f)) return;
        const float ion = 1.0f / sqrtf(o2);
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int e = 0; e < 3; ++e)
                if (act[d] && act[e]) J[3 * d + e] = s[d] * s[e] * ((d == e ? 1.f : 0.f) - o[d] * o[e] * ion * ion) * ion;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// --------------------------------------------------------------- G2P

// From the adjoint of (x', v', C', F') of each particle to the adjoint of the
// grid velocities (scattered into Gb.yzw) and G2P's part of the adjoint of
// (x, F); v and C do not enter G2P, so their adjoints are cleared here.
__global__ void __launch_bounds__(kThreads) k_adj_g2p(DevParams P, PState S, uint32_t n,
                                                       const float4 *__restrict__ Gv, AdjState A,
                                                       float4 *__restrict__ Gb) {
    const float dx = P.dx, K = 4.0f * P.inv_dx * P.inv_dx, dt = P.dt;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        uint32_t err = 0;
        const float4 xi = S.xi[s];
        int b[3];
        float f[3];
        f[0] = stencil_axis(xi.x, P.inv_dx, P.n, b[0], err);
        f[1] = stencil_axis(xi.y, P.inv_dx, P.n, b[1], err);
        f[2] = stencil_axis(xi.z, P.inv_dx, P.n, b[2], err);
        float w[3][3], dw[3][3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            bspline_weights(f[d], w[d]);
            bspline_slopes(f[d], dw[d]);
        }
        // forward: C' = (4/dx^2) sum w v (x_i - x_p)^T
        float Bm[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) Bm[q] = 0.f;
#pragma unroll 1
        for (int kk = 0; kk < 3; ++kk)
#pragma unroll
            for (int jj = 0; jj < 3; ++jj)
#pragma unroll
                for (int ii = 0; ii < 3; ++ii) {
                    const float wg = w[0][ii] * w[1][jj] * w[2][kk];
                    const float dp[3] = {(ii - f[0]) * dx, (jj - f[1]) * dx, (kk - f[2]) * dx};
                    const float4 g = Gv[node_addr(b[0] + ii, b[1] + jj, b[2] + kk, P.nb)];
                    const float vv[3] = {g.y, g.z, g.w};
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int c = 0; c < 3; ++c) Bm[3 * a + c] += wg * vv[a] * dp[c];
                }
        const float4 a0 = S.f0[s], a1 = S.f1[s];
        const float F[9] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, S.f2[s]};
        float xbo[3], vbo[3], Cbo[9], Fbo[9];
#pragma unroll
        for (int a = 0; a < 3; ++a) { xbo[a] = A.x[3 * (size_t)s + a]; vbo[a] = A.v[3 * (size_t)s + a]; }
#pragma unroll
        for (int q = 0; q < 9; ++q) { Cbo[q] = A.C[9 * (size_t)s + q]; Fbo[q] = A.F[9 * (size_t)s + q]; }
        float vbt[3], xbn[3], Cbt[9], Fbn[9];
#pragma unroll
        for (int a = 0; a < 3; ++a) { vbt[a] = vbo[a] + dt * xbo[a]; xbn[a] = xbo[a]; }   // x' = x + dt v'
#pragma unroll
        for (int a = 0; a < 3; ++a)                                                       // F' = (I + dt C') F
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float sF = Fbo[3 * a + c], sC = 0.f;
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    sF += dt * K * Bm[3 * e + a] * Fbo[3 * e + c];
                    sC += Fbo[3 * a + e] * F[3 * c + e];
                }
                Fbn[3 * a + c] = sF;
                Cbt[3 * a + c] = Cbo[3 * a + c] + dt * sC;
            }
#pragma unroll 1
        for (int kk = 0; kk < 3; ++kk)
#pragma unroll
            for (int jj = 0; jj < 3; ++jj)
#pragma unroll
                for (int ii = 0; ii < 3; ++ii) {
                    const float wg = w[0][ii] * w[1][jj] * w[2][kk];
                    const float gw[3] = {dw[0][ii] * w[1][jj] * w[2][kk] * P.inv_dx,
                                         w[0][ii] * dw[1][jj] * w[2][kk] * P.inv_dx,
                                         w[0][ii] * w[1][jj] * dw[2][kk] * P.inv_dx};
                    const float dp[3] = {(ii - f[0]) * dx, (jj - f[1]) * dx, (kk - f[2]) * dx};
                    const uint32_t I = node_addr(b[0] + ii, b[1] + jj, b[2] + kk, P.nb);
                    const float4 g = Gv[I];
                    const float vv[3] = {g.y, g.z, g.w};
                    float val[3], sdot = 0.f;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float cd = Cbt[3 * a] * dp[0] + Cbt[3 * a + 1] * dp[1] + Cbt[3 * a + 2] * dp[2];
                        val[a] = vbt[a] + K * cd;                    // Eqs. 8-9
                        sdot += vv[a] * val[a];
                    }
                    atomicAdd(&Gb[I], make_float4(0.f, wg * val[0], wg * val[1], wg * val[2]));
#pragma unroll
                    for (int c = 0; c < 3; ++c)                      // d (x_i - x_p) / d x_p = -I
                        xbn[c] += gw[c] * sdot - K * wg * (Cbt[c] * vv[0] + Cbt[3 + c] * vv[1] + Cbt[6 + c] * vv[2]);
                }
#pragma unroll
        for (int a = 0; a < 3; ++a) { A.x[3 * (size_t)s + a] = xbn[a]; A.v[3 * (size_t)s + a] = 0.f; }
#pragma unroll
        for (int q = 0; q < 9; ++q) { A.F[9 * (size_t)s + q] = Fbn[q]; A.C[9 * (size_t)s + q] = 0.f; }
    }
}

// ------------------------------------------------------ grid operation

// Gb.yzw holds dL/d(grid velocity) on entry; on return Gb = (dL/dm, dL/dmv).
// G holds the grid (m, mv) the forward grid operation read.  tool_bar
// (ntools x 18: R row-major, T, u, w) accumulates dL/d(frame entries).
__global__ void __launch_bounds__(kThreads) k_adj_grid(DevParams P, const float4 *__restrict__ G,
                                                        const ToolFrame *__restrict__ tools,
                                                        float4 *__restrict__ Gb, double *__restrict__ tool_bar) {
    __shared__ ToolFrame s_tools[kMaxTools];
    const int ntools = P.envp[0].ntools;
    if (threadIdx.x < ntools * (sizeof(ToolFrame) / 4))
        reinterpret_cast<float *>(s_tools)[threadIdx.x] = reinterpret_cast<const float *>(tools)[threadIdx.x];
    __syncthreads();
    const uint32_t total = (uint32_t)P.n * P.n * P.n;   // a multiple of 512: whole warps stay in the loop
    const int lo = P.bound, hi = P.n - P.bound;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        const float4 node = G[g];
        const float4 gb = Gb[g];
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
}

// ---------------------------------------------------------------- P2G

// From Gb = (dL/dm, dL/dmv) to the adjoint of (x, v, C, F): adds to G2P's
// parts in A.x and A.F, writes A.v and A.C; lame_bar[2] accumulates
// dL/dmu, dL/dlambda.
__global__ void __launch_bounds__(kThreads) k_adj_p2g(DevParams P, PState S, VCState V, uint32_t n,
                                                       const float4 *__restrict__ Gb, AdjState A,
                                                       double *__restrict__ lame_bar) {
    const EnvParams ep = P.envp[0];
    const float dx = P.dx, m = ep.mass, sk = ep.stress_k;
    float mub = 0.f, lamb = 0.f;
    const uint32_t span = (n + 31u) & ~31u;            // whole warps for the reduction
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < span; s += gridDim.x * blockDim.x) {
        if (s < n) {
            uint32_t err = 0;
            const float4 xi = S.xi[s];
            const float4 a0 = S.f0[s], a1 = S.f1[s];
            const float F[9] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, S.f2[s]};
            const float4 c0 = V.vc0[s], c1 = V.vc1[s], c2 = V.vc2[s];
            const float vp[3] = {c0.x, c0.y, c0.z};
            const float C[9] = {c0.w, c1.x, c1.y, c1.z, c1.w, c2.x, c2.y, c2.z, c2.w};
            float t6[6];
            kirchhoff(F, ep.mu, ep.lam, t6, err);
            const float tau[9] = {t6[0], t6[1], t6[2], t6[1], t6[3], t6[4], t6[2], t6[4], t6[5]};
            float Am[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) Am[q] = m * C[q] - sk * tau[q];     // A = m C - dt V0 (4/dx^2) tau
            int b[3];
            float f[3];
            f[0] = stencil_axis(xi.x, P.inv_dx, P.n, b[0], err);
            f[1] = stencil_axis(xi.y, P.inv_dx, P.n, b[1], err);
            f[2] = stencil_axis(xi.z, P.inv_dx, P.n, b[2], err);
            float w[3][3], dw[3][3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                bspline_weights(f[d], w[d]);
                bspline_slopes(f[d], dw[d]);
            }
            float Ab[9], vbp[3] = {0.f, 0.f, 0.f}, xbp[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < 9; ++q) Ab[q] = 0.f;
#pragma unroll 1
            for (int kk = 0; kk < 3; ++kk)
#pragma unroll
                for (int jj = 0; jj < 3; ++jj)
#pragma unroll
                    for (int ii = 0; ii < 3; ++ii) {
                        const float wg = w[0][ii] * w[1][jj] * w[2][kk];
                        const float gw[3] = {dw[0][ii] * w[1][jj] * w[2][kk] * P.inv_dx,
                                             w[0][ii] * dw[1][jj] * w[2][kk] * P.inv_dx,
                                             w[0][ii] * w[1][jj] * dw[2][kk] * P.inv_dx};
                        const float dp[3] = {(ii - f[0]) * dx, (jj - f[1]) * dx, (kk - f[2]) * dx};
                        const float4 g = Gb[node_addr(b[0] + ii, b[1] + jj, b[2] + kk, P.nb)];
                        const float mvb[3] = {g.y, g.z, g.w};
                        float sdot = g.x * m;
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            const float mom = m * vp[a] + Am[3 * a] * dp[0] + Am[3 * a + 1] * dp[1] + Am[3 * a + 2] * dp[2];
                            sdot += mvb[a] * mom;
                            vbp[a] += m * wg * mvb[a];
#pragma unroll
                            for (int c = 0; c < 3; ++c) Ab[3 * a + c] += wg * mvb[a] * dp[c];
                        }
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            xbp[c] += gw[c] * sdot - wg * (Am[c] * mvb[0] + Am[3 + c] * mvb[1] + Am[6 + c] * mvb[2]);
                    }
            // tau = mu (F F^T - I) + lambda ln(J) I
            float taub[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) taub[q] = -sk * Ab[q];
            const float trb = taub[0] + taub[4] + taub[8];
            const float cof[9] = {F[4] * F[8] - F[5] * F[7], F[5] * F[6] - F[3] * F[8], F[3] * F[7] - F[4] * F[6],
                                  F[2] * F[7] - F[1] * F[8], F[0] * F[8] - F[2] * F[6], F[1] * F[6] - F[0] * F[7],
                                  F[1] * F[5] - F[2] * F[4], F[2] * F[3] - F[0] * F[5], F[0] * F[4] - F[1] * F[3]};
            const float J = F[0] * cof[0] + F[1] * cof[1] + F[2] * cof[2];
            const float lnJ = logf(J > 0.f ? J : 1e-6f);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float fbb = ep.mu * ((taub[3 * a] + taub[a]) * F[c] + (taub[3 * a + 1] + taub[3 + a]) * F[3 + c] +
                                               (taub[3 * a + 2] + taub[6 + a]) * F[6 + c]);
                    const float fbl = J > 0.f ? ep.lam * trb * cof[3 * a + c] / J : 0.f;   // F^-T = cof(F) / J
                    A.F[9 * (size_t)s + 3 * a + c] += fbb + fbl;
                    mub += taub[3 * a + c] * ((F[3 * a] * F[3 * c] + F[3 * a + 1] * F[3 * c + 1] +
                                               F[3 * a + 2] * F[3 * c + 2]) - (a == c ? 1.f : 0.f));
                }
            lamb += trb * lnJ;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                A.x[3 * (size_t)s + a] += xbp[a];
                A.v[3 * (size_t)s + a] = vbp[a];
            }
#pragma unroll
            for (int q = 0; q < 9; ++q) A.C[9 * (size_t)s + q] = m * Ab[q];
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
                    int grid, cudaStream_t st) {
    if (n == 0) return;
    k_adj_g2p<<<grid, kThreads, 0, st>>>(P, S, n, Gv, A, Gb);
}
void launch_adj_grid(const DevParams &P, const float4 *G, const ToolFrame *tools, float4 *Gb, double *tool_bar,
                     int grid, cudaStream_t st) {
    k_adj_grid<<<grid, kThreads, 0, st>>>(P, G, tools, Gb, tool_bar);
}
void launch_adj_p2g(const DevParams &P, const PState &S, const VCState &V, uint32_t n, const float4 *Gb,
                    const AdjState &A, double *lame_bar, int grid, cudaStream_t st) {
    if (n == 0) return;
    k_adj_p2g<<<grid, kThreads, 0, st>>>(P, S, V, n, Gb, A, lame_bar);
}

}  // namespace gbmpm
