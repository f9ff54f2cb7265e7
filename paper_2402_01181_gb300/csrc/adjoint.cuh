// adjoint.cuh -- per-particle reverse mode of G2P (Eqs. 4, 8-10) and P2G
// (Eqs. 1-3 with the stress of Eqs. 5-6), shared by the unsorted adjoint
// kernels (particles in load order, global grid) and the block-sorted reverse
// sub-step (shared-memory tiles).  Node values are reached through accessors,
// so one arithmetic serves both.  Every branch of the forward pass is held at
// the side it took.
#pragma once

#include "common.cuh"

namespace gbmpm {

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

// a[k] for a run-time k in 0..2 by selects, so that a stays in registers
template <class T>
__device__ __forceinline__ T pick3(const T a[3], int k) { return k == 0 ? a[0] : (k == 1 ? a[1] : a[2]); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}


// Sums of per-particle partials over the lanes that share a particle: the
// identity when one thread handles the whole stencil.
struct OneLane {
    __device__ __forceinline__ float operator()(float v) const { return v; }
};
// Three lanes l0, l0+1, l0+2 of a warp, one z-plane of the stencil each; every
// lane gets the same sum (added in a fixed order).  Called by all 32 lanes.
struct ThreeLanes {
    int l0;
    __device__ __forceinline__ float operator()(float v) const {
        const float a = __shfl_sync(0xffffffffu, v, l0), b = __shfl_sync(0xffffffffu, v, l0 + 1),
                    c = __shfl_sync(0xffffffffu, v, l0 + 2);
        return (a + b) + c;
    }
};

// Per-axis stencil tables of one particle: weights w, their gradients dw in
// world units (d w / d x), and node offsets dp = (i - f) dx from the particle.
struct StencilAxes {
    int b[3];
    float f[3], w[3][3], dw[3][3], dp[3][3];
};
__device__ __forceinline__ void stencil_axes(const DevParams &P, const float xp[3], StencilAxes &S) {
    uint32_t err = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        S.f[d] = stencil_axis(xp[d], P.inv_dx, P.n, S.b[d], err);
        bspline_weights(S.f[d], S.w[d]);
        bspline_slopes(S.f[d], S.dw[d]);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            S.dw[d][i] *= P.inv_dx;
            S.dp[d][i] = ((float)i - S.f[d]) * P.dx;
        }
    }
}

// Reverse of G2P and advection for one particle (state x, F before the
// sub-step; V(ii, jj, kk) the grid velocity at its stencil nodes).  From the
// adjoint of the state after the sub-step (xbo, vbo, Cbo, Fbo) it hands the
// velocity adjoint of every stencil node to scatter(ii, jj, kk, value) and
// returns G2P's part of the adjoint of x and F (v and C do not enter G2P).
// The stencil's z-planes kk0 .. kk0+nkk-1 are this thread's; red sums the
// partials over the threads that share the particle (FULL: all three, with the
// z-planes unrolled, for callers whose node accessors load from global
// memory).  Cnew and vnew, if both
// given, are the particle's C and v after the sub-step (kept by the forward
// pass), which spares the recomputation of Eqs. 8-9's sums.
//
// With val_i = vbar + K Cbar (x_i - x_p) (K = 4/dx^2, vbar and Cbar the
// adjoints of v and C including advection and the F update), node i gets
// w_i val_i.  The adjoint of x_p is sum_i grad w_i (V_i . val_i) from the
// weights, plus -K Cbar^T sum_i w_i V_i = -K Cbar^T v from the offsets
// x_i - x_p, since sum_i w_i V_i is the particle's new velocity (Eq. 8).
template <class VelAt, class Scatter, class Red = OneLane, bool FULL = false>
__device__ __forceinline__ void adj_g2p_particle(const DevParams &P, const float xp[3], const float F[9], VelAt vel,
                                                 const float xbo[3], const float vbo[3], const float Cbo[9],
                                                 const float Fbo[9], Scatter scatter, float xbn[3], float Fbn[9],
                                                 int kk0 = 0, int nkk = 3, Red red = Red(),
                                                 const float *Cnew = nullptr, const float *vnew = nullptr) {
    const float K = 4.0f * P.inv_dx * P.inv_dx, dt = P.dt;
    StencilAxes S;
    stencil_axes(P, xp, S);
    // forward: C' = (4/dx^2) sum w v (x_i - x_p)^T, v' = sum w v
    float KB[9], vp[3];          // C' and v' themselves
    const bool kept = Cnew != nullptr && vnew != nullptr;
    if (kept) {
#pragma unroll
        for (int q = 0; q < 9; ++q) KB[q] = Cnew[q];
#pragma unroll
        for (int a = 0; a < 3; ++a) vp[a] = vnew[a];
    } else {
        float Bm[9], vs[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 9; ++q) Bm[q] = 0.f;
#pragma unroll(FULL ? 3 : 1)
        for (int kk = FULL ? 0 : kk0; kk < (FULL ? 3 : kk0 + nkk); ++kk) {
            const float wz = pick3(S.w[2], kk), dz = pick3(S.dp[2], kk);
#pragma unroll
            for (int jj = 0; jj < 3; ++jj)
#pragma unroll
                for (int ii = 0; ii < 3; ++ii) {
                    const float wg = S.w[0][ii] * S.w[1][jj] * wz;
                    const float dp[3] = {S.dp[0][ii], S.dp[1][jj], dz};
                    const float3 g = vel(S.b[0], S.b[1], S.b[2], ii, jj, kk);
                    const float vv[3] = {g.x, g.y, g.z};
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        vs[a] += wg * vv[a];
#pragma unroll
                        for (int c = 0; c < 3; ++c) Bm[3 * a + c] += wg * vv[a] * dp[c];
                    }
                }
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) KB[q] = K * red(Bm[q]);
#pragma unroll
        for (int a = 0; a < 3; ++a) vp[a] = red(vs[a]);
    }
    float vbt[3], Cbt[9];
#pragma unroll
    for (int a = 0; a < 3; ++a) vbt[a] = vbo[a] + dt * xbo[a];                       // x' = x + dt v'
#pragma unroll
    for (int a = 0; a < 3; ++a)                                                       // F' = (I + dt C') F
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float sF = Fbo[3 * a + c], sC = 0.f;
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                sF += dt * KB[3 * e + a] * Fbo[3 * e + c];
                sC += Fbo[3 * a + e] * F[3 * c + e];
            }
            Fbn[3 * a + c] = sF;
            Cbt[3 * a + c] = Cbo[3 * a + c] + dt * sC;
        }
    float Kc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) Kc[q] = K * Cbt[q];
    float xnode[3] = {0.f, 0.f, 0.f};
#pragma unroll(FULL ? 3 : 1)
    for (int kk = FULL ? 0 : kk0; kk < (FULL ? 3 : kk0 + nkk); ++kk) {
        const float wz = pick3(S.w[2], kk), dwz = pick3(S.dw[2], kk), dz = pick3(S.dp[2], kk);
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
            const float wyz = S.w[1][jj] * wz, dwyz = S.dw[1][jj] * wz, wydz = S.w[1][jj] * dwz;
            const float dy = S.dp[1][jj];
            float rv[3];                                           // val along the row, less its x part
#pragma unroll
            for (int a = 0; a < 3; ++a) rv[a] = fmaf(Kc[3 * a + 2], dz, fmaf(Kc[3 * a + 1], dy, vbt[a]));
            // the weight-gradient terms of the row: sum_ii dw_x sdot and sum_ii w_x sdot
            float sdw = 0.f, sw = 0.f;
#pragma unroll
            for (int ii = 0; ii < 3; ++ii) {
                const float wg = S.w[0][ii] * wyz;
                const float3 g = vel(S.b[0], S.b[1], S.b[2], ii, jj, kk);
                const float d0 = S.dp[0][ii];
                const float v0 = fmaf(Kc[0], d0, rv[0]), v1 = fmaf(Kc[3], d0, rv[1]), v2 = fmaf(Kc[6], d0, rv[2]);
                const float sdot = fmaf(g.z, v2, fmaf(g.y, v1, g.x * v0));      // Eqs. 8-9
                scatter(S.b[0], S.b[1], S.b[2], ii, jj, kk, make_float3(wg * v0, wg * v1, wg * v2));
                sdw = fmaf(S.dw[0][ii], sdot, sdw);
                sw = fmaf(S.w[0][ii], sdot, sw);
            }
            xnode[0] = fmaf(wyz, sdw, xnode[0]);
            xnode[1] = fmaf(dwyz, sw, xnode[1]);
            xnode[2] = fmaf(wydz, sw, xnode[2]);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)                                  // d (x_i - x_p) / d x_p = -I
        xbn[c] = xbo[c] + red(xnode[c]) - K * (Cbt[c] * vp[0] + Cbt[3 + c] * vp[1] + Cbt[6 + c] * vp[2]);
}

// Reverse of P2G for one particle (state x, v, C, F; Gb(ii, jj, kk) the
// adjoint (dL/dm, dL/dmv) of its stencil nodes).  Adds P2G's part to xb and
// Fb, returns the adjoint of v and C, and adds to mub, lamb the particle's
// part of dL/dmu and dL/dlambda (only if lead: one of the threads that share
// the particle).  The stencil's z-planes kk0 .. kk0+nkk-1 are this thread's;
// red sums the partials over the threads that share the particle (FULL: all
// three, unrolled).
//
// Node i receives w_i (m, m v + A (x_i - x_p)) with A = m C - dt V0 (4/dx^2) tau.
// With S = sum_i w_i mvbar_i: vbar = m S, Abar = sum_i w_i mvbar_i (x_i - x_p)^T,
// and the adjoint of x_p is sum_i grad w_i (mbar_i m + mvbar_i . mom_i) from the
// weights plus -A^T S from the offsets.
template <class GbarAt, class Red = OneLane, bool FULL = false>
__device__ __forceinline__ void adj_p2g_particle(const DevParams &P, const EnvParams &ep, const float xp[3],
                                                 const float vp[3], const float C[9], const float F[9], GbarAt gbar,
                                                 float xb[3], float Fb[9], float vb[3], float Cb[9], float &mub,
                                                 float &lamb, int kk0 = 0, int nkk = 3, Red red = Red(),
                                                 bool lead = true) {
    uint32_t err = 0;
    const float m = ep.mass, sk = ep.stress_k;
    float t6[6];
    kirchhoff(F, ep.mu, ep.lam, t6, err);
    const float tau[9] = {t6[0], t6[1], t6[2], t6[1], t6[3], t6[4], t6[2], t6[4], t6[5]};
    float Am[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) Am[q] = m * C[q] - sk * tau[q];     // A = m C - dt V0 (4/dx^2) tau
    StencilAxes S;
    stencil_axes(P, xp, S);
    const float mv[3] = {m * vp[0], m * vp[1], m * vp[2]};
    float Ab[9], Sm[3] = {0.f, 0.f, 0.f}, xbp[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 9; ++q) Ab[q] = 0.f;
#pragma unroll(FULL ? 3 : 1)
    for (int kk = FULL ? 0 : kk0; kk < (FULL ? 3 : kk0 + nkk); ++kk) {
        const float wz = pick3(S.w[2], kk), dwz = pick3(S.dw[2], kk), dz = pick3(S.dp[2], kk);
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
            const float wyz = S.w[1][jj] * wz, dwyz = S.dw[1][jj] * wz, wydz = S.w[1][jj] * dwz;
            const float dy = S.dp[1][jj];
            float rm[3], R0[3] = {0.f, 0.f, 0.f}, R1[3] = {0.f, 0.f, 0.f}, sdw = 0.f, sw = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a) rm[a] = fmaf(Am[3 * a + 2], dz, fmaf(Am[3 * a + 1], dy, mv[a]));
#pragma unroll
            for (int ii = 0; ii < 3; ++ii) {
                const float wg = S.w[0][ii] * wyz;
                const float4 g = gbar(S.b[0], S.b[1], S.b[2], ii, jj, kk);
                const float d0 = S.dp[0][ii];
                const float mvb[3] = {g.y, g.z, g.w};
                float sdot = g.x * m;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    sdot = fmaf(mvb[a], fmaf(Am[3 * a], d0, rm[a]), sdot);     // mom_i
                    const float t = wg * mvb[a];
                    R0[a] += t;
                    R1[a] = fmaf(t, d0, R1[a]);
                }
                sdw = fmaf(S.dw[0][ii], sdot, sdw);
                sw = fmaf(S.w[0][ii], sdot, sw);
            }
            xbp[0] = fmaf(wyz, sdw, xbp[0]);
            xbp[1] = fmaf(dwyz, sw, xbp[1]);
            xbp[2] = fmaf(wydz, sw, xbp[2]);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                Ab[3 * a] += R1[a];
                Ab[3 * a + 1] = fmaf(R0[a], dy, Ab[3 * a + 1]);
                Ab[3 * a + 2] = fmaf(R0[a], dz, Ab[3 * a + 2]);
                Sm[a] += R0[a];
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) Ab[q] = red(Ab[q]);
#pragma unroll
    for (int a = 0; a < 3; ++a) Sm[a] = red(Sm[a]);
    float vbp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        xbp[c] = red(xbp[c]) - (Am[c] * Sm[0] + Am[3 + c] * Sm[1] + Am[6 + c] * Sm[2]);
        vbp[c] = m * Sm[c];
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
            Fb[3 * a + c] += fbb + fbl;
            if (lead)
                mub += taub[3 * a + c] * ((F[3 * a] * F[3 * c] + F[3 * a + 1] * F[3 * c + 1] +
                                           F[3 * a + 2] * F[3 * c + 2]) - (a == c ? 1.f : 0.f));
        }
    if (lead) lamb += trb * lnJ;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xb[a] += xbp[a];
        vb[a] = vbp[a];
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) Cb[q] = m * Ab[q];
}

}  // namespace gbmpm
