// kernels_split.cu -- the separate-kernel MLS-MPM sub-step (P2G scatter with
// global atomics, grid operation over all nodes, G2P) plus the load, readout
// and grid-inspection kernels both pipelines use.
#include "common.cuh"
#include "launch.h"

namespace gbmpm {

// ---------------------------------------------------------------- P2G

// P2G of one particle (Eqs. 1-3): scatters w_ip (m_p, m_p v_p + A_p (x_i - x_p))
// with A_p = m_p C_p - dt V_p^0 (4/dx^2) tau(F_p) into the blocked grid with
// float4 atomics.
__global__ void __launch_bounds__(256) k_p2g_scatter(DevParams P, PState S, VCState V, uint32_t n,
                                                      float4 *__restrict__ G, Ctrl *ctrl) {
    uint32_t err = 0;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const float4 xi = S.xi[s];
        const float4 a0 = S.f0[s], a1 = S.f1[s];
        const float F[9] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, S.f2[s]};
        const float4 c0 = V.vc0[s], c1 = V.vc1[s], c2 = V.vc2[s];
        const float C[9] = {c0.w, c1.x, c1.y, c1.z, c1.w, c2.x, c2.y, c2.z, c2.w};
        const uint32_t e = P.n_envs > 1 ? env_of_particle(__float_as_uint(xi.w), P) : 0u;
        const EnvParams ep = P.envp[e];
        float t[6];
        kirchhoff(F, ep.mu, ep.lam, t, err);
        if (!finite3(xi.x, xi.y, xi.z) || !finite3(c0.x, c0.y, c0.z)) err |= kErrNumeric;
        const float m = ep.mass, k = ep.stress_k;
        // A scaled by dx (so that A (x_i - x_p) = A' (o - fx))
        const float A[9] = {(m * C[0] - k * t[0]) * P.dx, (m * C[1] - k * t[1]) * P.dx, (m * C[2] - k * t[2]) * P.dx,
                            (m * C[3] - k * t[1]) * P.dx, (m * C[4] - k * t[3]) * P.dx, (m * C[5] - k * t[4]) * P.dx,
                            (m * C[6] - k * t[2]) * P.dx, (m * C[7] - k * t[4]) * P.dx, (m * C[8] - k * t[5]) * P.dx};
        int bx, by, bz;
        const float fx = stencil_axis(xi.x, P.inv_dx, P.n, bx, err);
        const float fy = stencil_axis(xi.y, P.inv_dx, P.n, by, err);
        const float fz = stencil_axis(xi.z, P.inv_dx, P.n, bz, err);
        float wx[3], wy[3], wz[3];
        bspline_weights(fx, wx);
        bspline_weights(fy, wy);
        bspline_weights(fz, wz);
        // q = m v - A' fx : value at offset o is q + A' o
        const float qx = m * c0.x - (A[0] * fx + A[1] * fy + A[2] * fz);
        const float qy = m * c0.y - (A[3] * fx + A[4] * fy + A[5] * fz);
        const float qz = m * c0.z - (A[6] * fx + A[7] * fy + A[8] * fz);
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) {
                const float wjk = wy[jj] * wz[kk];
                const float rx = qx + A[1] * jj + A[2] * kk;
                const float ry = qy + A[4] * jj + A[5] * kk;
                const float rz = qz + A[7] * jj + A[8] * kk;
#pragma unroll
                for (int ii = 0; ii < 3; ++ii) {
                    const float w = wx[ii] * wjk;
                    const float4 val = make_float4(w * m, w * (rx + A[0] * ii), w * (ry + A[3] * ii), w * (rz + A[6] * ii));
                    atomicAdd(&G[node_addr_env(e, bx + ii, by + jj, bz + kk, P.nb, P.nbe)], val);
                }
            }
        }
    }
    if (err) atomicOr(&ctrl->err, err);
}

// ------------------------------------------------------ grid operation

// Gout may equal Gin (in place).
__global__ void __launch_bounds__(256) k_grid_update_dense(DevParams P, const float4 *Gin, float4 *Gout,
                                                            const ToolFrame *__restrict__ tools) {
    __shared__ ToolFrame s_tools[kMaxTools];
    const int ntools = P.envp[0].ntools;
    if (threadIdx.x < ntools * (sizeof(ToolFrame) / 4))
        reinterpret_cast<float *>(s_tools)[threadIdx.x] = reinterpret_cast<const float *>(tools)[threadIdx.x];
    __syncthreads();
    const uint32_t total = (uint32_t)P.n * P.n * P.n;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        const float4 node = Gin[g];
        if (!(node.x > 0.0f)) {
            if (Gout != Gin || node.y != 0.f || node.z != 0.f || node.w != 0.f) Gout[g] = make_float4(node.x, 0.f, 0.f, 0.f);
            continue;
        }
        const uint32_t b = g >> 6, l = g & 63u;
        const int bx = b % P.nb, by = (b / P.nb) % P.nb, bz = b / (P.nb * P.nb);
        const int i = bx * 4 + (l & 3), j = by * 4 + ((l >> 2) & 3), k = bz * 4 + (l >> 4);
        const float3 v = grid_node_update(node.x, node.y, node.z, node.w, i, j, k, P, s_tools, ntools);
        Gout[g] = make_float4(node.x, v.x, v.y, v.z);
    }
}

// ------------------------------------------------------------------ G2P

// G2P and advection of one particle (Eqs. 8-10) with the F update of Eq. 4,
// reading grid velocities stored in place of the momentum.
__global__ void __launch_bounds__(256) k_g2p_split(DevParams P, PState S, VCState V, uint32_t n,
                                                    const float4 *__restrict__ G, Ctrl *ctrl) {
    uint32_t err = 0;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const float4 xi = S.xi[s];
        int bx, by, bz;
        const float fx = stencil_axis(xi.x, P.inv_dx, P.n, bx, err);
        const float fy = stencil_axis(xi.y, P.inv_dx, P.n, by, err);
        const float fz = stencil_axis(xi.z, P.inv_dx, P.n, bz, err);
        float wx[3], wy[3], wz[3];
        bspline_weights(fx, wx);
        bspline_weights(fy, wy);
        bspline_weights(fz, wz);
        float vx = 0.f, vy = 0.f, vz = 0.f;
        float B[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // sum w v (o - f)^T
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) {
                const float wjk = wy[jj] * wz[kk];
                float ax = 0.f, ay = 0.f, az = 0.f, bxx = 0.f, bxy = 0.f, bxz = 0.f;
#pragma unroll
                for (int ii = 0; ii < 3; ++ii) {
                    const float4 g = G[node_addr(bx + ii, by + jj, bz + kk, P.nb)];
                    const float wi = wx[ii], wo = wx[ii] * (ii - fx);
                    ax += wi * g.y; ay += wi * g.z; az += wi * g.w;
                    bxx += wo * g.y; bxy += wo * g.z; bxz += wo * g.w;
                }
                const float dy = wjk * (jj - fy), dz = wjk * (kk - fz);
                vx += wjk * ax; vy += wjk * ay; vz += wjk * az;
                B[0] += wjk * bxx; B[3] += wjk * bxy; B[6] += wjk * bxz;
                B[1] += dy * ax; B[4] += dy * ay; B[7] += dy * az;
                B[2] += dz * ax; B[5] += dz * ay; B[8] += dz * az;
            }
        }
        const float cs = 4.0f * P.inv_dx;      // 4/dx^2 * dx
        float C[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) C[q] = cs * B[q];
        const float4 a0 = S.f0[s], a1 = S.f1[s];
        const float F[9] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, S.f2[s]};
        float Fn[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                Fn[3 * r + c] = F[3 * r + c] + P.dt * (C[3 * r] * F[c] + C[3 * r + 1] * F[3 + c] + C[3 * r + 2] * F[6 + c]);
        const float nx = xi.x + P.dt * vx, ny = xi.y + P.dt * vy, nz = xi.z + P.dt * vz;
        if (!finite3(nx, ny, nz) || !finite3(vx, vy, vz)) err |= kErrNumeric;
        S.xi[s] = make_float4(nx, ny, nz, xi.w);
        S.f0[s] = make_float4(Fn[0], Fn[1], Fn[2], Fn[3]);
        S.f1[s] = make_float4(Fn[4], Fn[5], Fn[6], Fn[7]);
        S.f2[s] = Fn[8];
        store_vc(V, s, vx, vy, vz, C);
    }
    if (err) atomicOr(&ctrl->err, err);
}

// ---------------------------------------------------------- load / read

// Load n particles in index order into slots 0..n-1 (ids = slots).
__global__ void k_load_identity(const float *__restrict__ x, const float *__restrict__ v, const float *__restrict__ F,
                                const float *__restrict__ C, uint32_t n, PState S, VCState V, Ctrl *ctrl) {
    uint32_t err = 0;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float px = x[3 * p], py = x[3 * p + 1], pz = x[3 * p + 2];
        if (!finite3(px, py, pz)) err |= kErrNumeric;
        S.xi[p] = make_float4(px, py, pz, __uint_as_float(p));
        float f[9], c[9], vv[3];
        for (int q = 0; q < 9; ++q) {
            f[q] = F ? F[9 * (size_t)p + q] : ((q % 4) == 0 ? 1.0f : 0.0f);
            c[q] = C ? C[9 * (size_t)p + q] : 0.0f;
        }
        for (int q = 0; q < 3; ++q) vv[q] = v ? v[3 * (size_t)p + q] : 0.0f;
        S.f0[p] = make_float4(f[0], f[1], f[2], f[3]);
        S.f1[p] = make_float4(f[4], f[5], f[6], f[7]);
        S.f2[p] = f[8];
        store_vc(V, p, vv[0], vv[1], vv[2], c);
    }
    if (err) atomicOr(&ctrl->err, err);
}

// Write the state of slots 0..n-1 to row-major outputs indexed by particle id.
__global__ void k_read_out(PState S, VCState V, uint32_t n, float *__restrict__ x, float *__restrict__ v,
                           float *__restrict__ F, float *__restrict__ C) {
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const float4 xi = S.xi[s];
        const size_t p = __float_as_uint(xi.w);
        if (p >= n) continue;   // slot not filled (possible only after a capacity error)
        if (x) { x[3 * p] = xi.x; x[3 * p + 1] = xi.y; x[3 * p + 2] = xi.z; }
        if (F) {
            const float4 a0 = S.f0[s], a1 = S.f1[s];
            float *o = F + 9 * p;
            o[0] = a0.x; o[1] = a0.y; o[2] = a0.z; o[3] = a0.w;
            o[4] = a1.x; o[5] = a1.y; o[6] = a1.z; o[7] = a1.w; o[8] = S.f2[s];
        }
        if (v || C) {
            const float4 c0 = V.vc0[s], c1 = V.vc1[s], c2 = V.vc2[s];
            if (v) { v[3 * p] = c0.x; v[3 * p + 1] = c0.y; v[3 * p + 2] = c0.z; }
            if (C) {
                float *o = C + 9 * p;
                o[0] = c0.w; o[1] = c1.x; o[2] = c1.y; o[3] = c1.z;
                o[4] = c1.w; o[5] = c2.x; o[6] = c2.y; o[7] = c2.z; o[8] = c2.w;
            }
        }
    }
}

// Blocked grid -> dense [i][j][k] (k fastest) float4 rows.
__global__ void k_grid_to_dense(int n, int nb, int n_envs, const float4 *__restrict__ G, float4 *__restrict__ out) {
    const uint32_t per = (uint32_t)n * n * n, total = per * (uint32_t)n_envs;
    const uint32_t nbe = (uint32_t)nb * nb * nb;
    for (uint32_t d = blockIdx.x * blockDim.x + threadIdx.x; d < total; d += gridDim.x * blockDim.x) {
        const uint32_t e = d / per, r = d % per;
        const int k = r % n, j = (r / n) % n, i = r / (n * n);
        out[d] = G[node_addr_env(e, i, j, k, nb, nbe)];
    }
}

// Grid operation of every node of the blocked grids G (m, mv) of all
// environments into dense [e][i][j][k] velocity rows (3 floats); tools is the
// frame table of one sub-step (tstride frames per environment).
__global__ void k_grid_velocity_dense(DevParams P, const float4 *__restrict__ G, const ToolFrame *__restrict__ tools,
                                      float *__restrict__ out) {
    const int n = P.n;
    const uint32_t per = (uint32_t)n * n * n, total = per * (uint32_t)P.n_envs;
    for (uint32_t d = blockIdx.x * blockDim.x + threadIdx.x; d < total; d += gridDim.x * blockDim.x) {
        const uint32_t e = d / per, r = d % per;
        const int k = r % n, j = (r / n) % n, i = r / (n * n);
        const float4 g = G[node_addr_env(e, i, j, k, P.nb, P.nbe)];
        const float3 v = grid_node_update(g.x, g.y, g.z, g.w, i, j, k, P, tools + (size_t)e * P.tstride,
                                          P.envp[e].ntools);
        out[3 * (size_t)d] = v.x;
        out[3 * (size_t)d + 1] = v.y;
        out[3 * (size_t)d + 2] = v.z;
    }
}

// ------------------------------------------------------------- launchers

void launch_p2g_scatter(const DevParams &P, const PState &S, const VCState &V, uint32_t n, float4 *G, Ctrl *ctrl,
                        int grid, cudaStream_t st) {
    if (n == 0) return;
    k_p2g_scatter<<<grid, 256, 0, st>>>(P, S, V, n, G, ctrl);
}
void launch_grid_update_dense(const DevParams &P, float4 *G, const ToolFrame *tools, int grid, cudaStream_t st) {
    k_grid_update_dense<<<grid, 256, 0, st>>>(P, G, G, tools);
}
void launch_grid_update_dense_to(const DevParams &P, const float4 *Gin, float4 *Gout, const ToolFrame *tools, int grid,
                                 cudaStream_t st) {
    k_grid_update_dense<<<grid, 256, 0, st>>>(P, Gin, Gout, tools);
}
void launch_g2p_split(const DevParams &P, const PState &S, const VCState &V, uint32_t n, const float4 *G, Ctrl *ctrl,
                      int grid, cudaStream_t st) {
    if (n == 0) return;
    k_g2p_split<<<grid, 256, 0, st>>>(P, S, V, n, G, ctrl);
}
void launch_load_identity(const float *x, const float *v, const float *F, const float *C, uint32_t n, const PState &S,
                          const VCState &V, Ctrl *ctrl, int grid, cudaStream_t st) {
    if (n == 0) return;
    k_load_identity<<<grid, 256, 0, st>>>(x, v, F, C, n, S, V, ctrl);
}
void launch_read_out(const PState &S, const VCState &V, uint32_t n, float *x, float *v, float *F, float *C, int grid,
                     cudaStream_t st) {
    if (n == 0) return;
    k_read_out<<<grid, 256, 0, st>>>(S, V, n, x, v, F, C);
}
void launch_grid_to_dense(int n, int nb, int n_envs, const float4 *G, float4 *out, int grid, cudaStream_t st) {
    k_grid_to_dense<<<grid, 256, 0, st>>>(n, nb, n_envs, G, out);
}
void launch_grid_velocity_dense(const DevParams &P, const float4 *G, const ToolFrame *tools, float *out, int grid,
                                cudaStream_t st) {
    k_grid_velocity_dense<<<grid, 256, 0, st>>>(P, G, tools, out);
}

}  // namespace gbmpm
