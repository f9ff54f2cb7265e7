// common.cuh -- device data layouts and per-node / per-particle arithmetic of
// the MLS-MPM sub-step (Sec. III-B, III-C of arXiv 2402.01181), shared by the
// fused and split kernels of this library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbmpm {

constexpr int kMaxTools = 8;

// Sticky device error bits (Ctrl::err).
enum : uint32_t {
    kErrNumeric = 1u,    // non-finite state or det F <= 0
    kErrDomain = 2u,     // stencil clamped to the grid
    kErrCapacity = 4u,   // run-table or particle-count overflow
    kErrCfl = 8u,        // particle moved by more than one block in a sub-step
};

// Per-environment material, in a device table indexed by environment.
struct EnvParams {
    float mass;       // m_p = rho V_p^0
    float mu, lam;    // Lame parameters (Eq. 6)
    float stress_k;   // dt V_p^0 4/dx^2 : A_p = m_p C_p - stress_k tau_p
    int ntools;       // tool slots in use (highest active id + 1)
    int pad[3];
};

// Per-handle constants, passed by value to every kernel.  A handle holds
// n_envs independent environments on identical grids; grid block g of the
// whole handle is block g % nbe of environment g / nbe.
struct DevParams {
    int n;            // nodes per axis
    int nb;           // 4x4x4 blocks per axis (n / 4)
    uint32_t nbe;     // blocks per environment (nb^3)
    int n_envs;
    int bound;        // sticky wall band
    int tstride;      // tool frames per environment in a sub-step's frame table
    float dx, inv_dx, dt;
    float gx, gy, gz;
    float theta, fric;
    const EnvParams *envp;     // n_envs entries
    const uint32_t *env_off;   // n_envs + 1 particle-index offsets (environments are contiguous)
};

// One tool at one sub-step, in FP32 (computed on the host in FP64).
struct __align__(16) ToolFrame {
    float R[9];       // row-major; world = R ref + T
    float T[3];
    float u[3];       // linear velocity of T
    float w[3];       // angular velocity
    float dims[3];    // capsule: (radius, half-length, -); box: half extents;
                      // sampled: tool-frame position o of sample (0, 0, 0)
    float reach2;     // squared radius beyond which the node is surely not in contact
    int kind;         // 0 capsule, 1 box, 2 sampled distance field, -1 none
    int res;          // sampled: samples per axis
    float inv_h;      // sampled: 1 / sample spacing h
    const float *sdf; // sampled: res^3 distances, x fastest; sample (i, j, k) is the
                      // distance at o + h (i, j, k)
};
static_assert(sizeof(ToolFrame) == 28 * 4, "ToolFrame layout");

// Particle state streams.  Slot s holds one particle:
//   xi[s] = (x, y, z, id bits)   f0 = (F00 F01 F02 F10)   f1 = (F11 F12 F20 F21)   f2 = F22
// and, when written, vc0 = (vx vy vz C00)  vc1 = (C01 C02 C10 C11)  vc2 = (C12 C20 C21 C22).
struct PState {
    float4 *xi;
    float4 *f0;
    float4 *f1;
    float *f2;
};
struct VCState {
    float4 *vc0;
    float4 *vc1;
    float4 *vc2;
};

// A chunk is the output of one 256-particle pass of the fused kernel: its
// particles are stored grouped by destination direction d (0..26); run[d] =
// (first slot, count).
struct Chunk {
    uint2 run[27];
};
// Per source block: which chunks it wrote in the last sub-step.
struct BlockTab {
    uint32_t stamp;   // sub-step index the entry is valid for
    uint32_t first;   // first chunk index
    uint32_t npass;   // number of chunks
    uint32_t pad;
};

// Control words living in device memory.
// The counters every CTA of a fused launch updates sit on separate 128-byte
// lines, so that their atomics are served by different L2 slices at once.
struct Ctrl {
    uint32_t step;              // sub-step index (monotonic, starts at 1 after a load)
    uint32_t n_particles;
    uint32_t err;               // sticky error bits
    uint32_t pad0[29];
    uint32_t done;              // CTAs finished in the current fused launch
    uint32_t pad1[31];
    uint32_t work;              // next work item of the current fused launch
    uint32_t pad2[31];
    uint32_t part_alloc;        // particle slots handed out in the current launch
    uint32_t pad3[31];
    uint32_t chunk_alloc;       // chunk entries handed out in the current launch
    uint32_t pad4[31];
    // active-block list sizes by sub-step parity: [0] heavy blocks, listed from
    // the front, [1] light blocks, listed from the back (one 64-bit read)
    uint32_t nactive[2][2];
    uint32_t pad5[28];
    uint32_t nclear[3];         // grid clear-list sizes, by sub-step mod 3
    uint32_t pad6[29];
};
static_assert(sizeof(Ctrl) == 7 * 128, "Ctrl: one 128-byte line per counter group");

// ----------------------------------------------------------- grid layout

// Grid nodes are stored in 4x4x4 blocks (x fastest inside the block and
// across blocks); every node is a float4 (m, mv_x, mv_y, mv_z) before the
// grid operation.
// Programmatic dependent launch (a kernel launched with the programmatic
// stream serialization attribute): griddep_wait() blocks until the previous
// kernel in the stream has completed and its memory is visible;
// griddep_launch_dependents() lets the next such kernel be scheduled once every
// CTA of this one has called it (or exited).  Both are no-ops for a kernel
// launched without the attribute.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" :::); }
// Launch kernel as a programmatic dependent of the stream's previous kernel.
template <typename... K, typename... A>
inline void launch_dependent(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);   // a failure is left for cudaGetLastError
}

__host__ __device__ __forceinline__ uint32_t block_id(int bx, int by, int bz, int nb) {
    return (uint32_t)(bx + nb * (by + nb * bz));
}
__host__ __device__ __forceinline__ uint32_t node_addr(int i, int j, int k, int nb) {
    return block_id(i >> 2, j >> 2, k >> 2, nb) * 64u + (uint32_t)((i & 3) + 4 * ((j & 3) + 4 * (k & 3)));
}
// node (i,j,k) of environment e
__host__ __device__ __forceinline__ uint32_t node_addr_env(uint32_t e, int i, int j, int k, int nb, uint32_t nbe) {
    return e * nbe * 64u + node_addr(i, j, k, nb);
}

// Environment of global particle index p (environments occupy contiguous
// index ranges env_off[e] .. env_off[e+1]).
__device__ __forceinline__ uint32_t env_of_particle(uint32_t p, const DevParams &P) {
    int lo = 0, hi = P.n_envs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.env_off[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return (uint32_t)lo;
}

// ------------------------------------------------------------ arithmetic

// Quadratic B-spline weights of nodes base, base+1, base+2 for fx in [0.5, 1.5).
__device__ __forceinline__ void bspline_weights(float fx, float w[3]) {
    const float a = 1.5f - fx, b = fx - 1.0f, c = fx - 0.5f;
    w[0] = 0.5f * a * a;
    w[1] = 0.75f - b * b;
    w[2] = 0.5f * c * c;
}

// Stencil base of one coordinate with clamping to [0, n-3]; returns fx.
__device__ __forceinline__ float stencil_axis(float x, float inv_dx, int n, int &base, uint32_t &err) {
    const float s = x * inv_dx;
    int b = __float2int_rd(s - 0.5f);
    if (b < 0) { b = 0; err |= kErrDomain; }
    if (b > n - 3) { b = n - 3; err |= kErrDomain; }
    base = b;
    return s - (float)b;
}

// Kirchhoff stress tau = P(F) F^T of the Neo-Hookean first Piola stress
// P = mu (F - F^-T) + lam ln(J) F^-T (Eq. 5, F^-T reading):
// tau = mu (F F^T - I) + lam ln(J) I; symmetric, returned as
// (t00, t01, t02, t11, t12, t22).
__device__ __forceinline__ void kirchhoff(const float F[9], float mu, float lam, float t[6], uint32_t &err) {
    const float J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                    F[2] * (F[3] * F[7] - F[4] * F[6]);
    float Jc = J;
    if (!(J > 0.0f)) { Jc = 1e-6f; err |= kErrNumeric; }
    const float lnJ = logf(Jc);
    const float bb00 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
    const float bb01 = F[0] * F[3] + F[1] * F[4] + F[2] * F[5];
    const float bb02 = F[0] * F[6] + F[1] * F[7] + F[2] * F[8];
    const float bb11 = F[3] * F[3] + F[4] * F[4] + F[5] * F[5];
    const float bb12 = F[3] * F[6] + F[4] * F[7] + F[5] * F[8];
    const float bb22 = F[6] * F[6] + F[7] * F[7] + F[8] * F[8];
    const float iso = lam * lnJ - mu;
    t[0] = mu * bb00 + iso;
    t[1] = mu * bb01;
    t[2] = mu * bb02;
    t[3] = mu * bb11 + iso;
    t[4] = mu * bb12;
    t[5] = mu * bb22 + iso;
}

// Sampled distance field of Eqs. 12-14.  The cell index of a tool-frame
// point is floor((p - o) / h) per axis (Eq. 12 indexes by x_ref / h); the
// distance is that sample, the normal the central difference of the
// neighbouring samples (Eq. 14; one-sided at the faces of the volume),
// normalised.  Points outside the sampled volume are not in contact.
// Returns (distance, normal).  Kept out of line: it is taken only for nodes
// near a sampled tool and would otherwise raise the register count of every
// kernel that runs the grid operation.
static __device__ __noinline__ float4 sampled_sdf(const float *sdf, int res, float inv_h, float ox, float oy, float oz,
                                           float px, float py, float pz) {
    const float ux = floorf((px - ox) * inv_h), uy = floorf((py - oy) * inv_h), uz = floorf((pz - oz) * inv_h);
    const float top = (float)res;
    if (!(ux >= 0.f && uy >= 0.f && uz >= 0.f && ux < top && uy < top && uz < top))
        return make_float4(3.0e38f, 0.f, 1.f, 0.f);
    const int i = (int)ux, j = (int)uy, k = (int)uz;
    const size_t r = (size_t)res;
    auto at = [&](int a, int b, int c) { return __ldg(&sdf[((size_t)c * r + b) * r + a]); };
    const int im = max(i - 1, 0), ip = min(i + 1, res - 1);
    const int jm = max(j - 1, 0), jp = min(j + 1, res - 1);
    const int km = max(k - 1, 0), kp = min(k + 1, res - 1);
    // differences over 2 samples inside, 1 at a face; the common factor 1/h drops out
    const float gx = (at(ip, j, k) - at(im, j, k)) / (float)max(ip - im, 1);
    const float gy = (at(i, jp, k) - at(i, jm, k)) / (float)max(jp - jm, 1);
    const float gz = (at(i, j, kp) - at(i, j, km)) / (float)max(kp - km, 1);
    const float g2 = gx * gx + gy * gy + gz * gz;
    if (!(g2 > 0.f)) return make_float4(at(i, j, k), 0.f, 1.f, 0.f);
    const float il = 1.0f / sqrtf(g2);
    return make_float4(at(i, j, k), gx * il, gy * il, gz * il);
}

// Signed distance of a tool-frame point to a capsule (axis along y) or a box
// and the outward unit normal there (analytic stand-in for Eqs. 12-14).
__device__ __forceinline__ float tool_sdf(int kind, const float *dims, float px, float py, float pz,
                                          float &nx, float &ny, float &nz) {
    if (kind == 0) {
        const float c = fminf(fmaxf(py, -dims[1]), dims[1]);
        const float qy = py - c;
        const float L2 = px * px + qy * qy + pz * pz;
        if (L2 > 0.0f) {
            const float L = sqrtf(L2);
            nx = px / L; ny = qy / L; nz = pz / L;
            return L - dims[0];
        }
        nx = 0.0f; ny = 1.0f; nz = 0.0f;
        return -dims[0];
    }
    const float qx = fabsf(px) - dims[0], qy = fabsf(py) - dims[1], qz = fabsf(pz) - dims[2];
    const float ox = fmaxf(qx, 0.0f), oy = fmaxf(qy, 0.0f), oz = fmaxf(qz, 0.0f);
    const float o2 = ox * ox + oy * oy + oz * oz;
    if (o2 > 0.0f) {
        const float on = sqrtf(o2);
        nx = copysignf(ox / on, px < 0.0f ? -1.0f : 1.0f);
        ny = copysignf(oy / on, py < 0.0f ? -1.0f : 1.0f);
        nz = copysignf(oz / on, pz < 0.0f ? -1.0f : 1.0f);
        return on;
    }
    // inside: nearest face, lowest axis on ties
    int a = 0;
    float qm = qx;
    if (qy > qm) { a = 1; qm = qy; }
    if (qz > qm) { a = 2; qm = qz; }
    nx = ny = nz = 0.0f;
    if (a == 0) nx = px < 0.0f ? -1.0f : 1.0f;
    else if (a == 1) ny = py < 0.0f ? -1.0f : 1.0f;
    else nz = pz < 0.0f ? -1.0f : 1.0f;
    return qm;
}

// z-buffer of Sec. III-C at a world node position: the closest tool (lowest
// index on ties), its distance dmin, the unit normal n_ref and the node
// position p_ref in that tool's frame (Eq. 11).  Tools whose reach the node
// is beyond are skipped: their distance is surely >= theta.  Returns -1 if no
// tool is within reach.
__device__ __forceinline__ int nearest_tool(float xw, float yw, float zw, const ToolFrame *tools, int ntools,
                                            float &dmin, float &nbx, float &nby, float &nbz, float &pbx,
                                            float &pby, float &pbz) {
    dmin = 3.0e38f;
    nbx = nby = nbz = 0.f;
    pbx = pby = pbz = 0.f;
    int id = -1;
    for (int t = 0; t < ntools; ++t) {
        const ToolFrame &tf = tools[t];
        if (tf.kind < 0) continue;
        const float rx = xw - tf.T[0], ry = yw - tf.T[1], rz = zw - tf.T[2];
        if (rx * rx + ry * ry + rz * rz > tf.reach2) continue;   // surely d >= theta
        // Eq. 11: x_ref = R^T (x - T)
        const float px = tf.R[0] * rx + tf.R[3] * ry + tf.R[6] * rz;
        const float py = tf.R[1] * rx + tf.R[4] * ry + tf.R[7] * rz;
        const float pz = tf.R[2] * rx + tf.R[5] * ry + tf.R[8] * rz;
        float nx, ny, nz, d;
        if (tf.kind == 2) {
            const float4 s = sampled_sdf(tf.sdf, tf.res, tf.inv_h, tf.dims[0], tf.dims[1], tf.dims[2], px, py, pz);
            d = s.x; nx = s.y; ny = s.z; nz = s.w;
        } else {
            d = tool_sdf(tf.kind, tf.dims, px, py, pz, nx, ny, nz);
        }
        if (d < dmin) { dmin = d; id = t; nbx = nx; nby = ny; nbz = nz; pbx = px; pby = py; pbz = pz; }
    }
    return id;
}

// Grid operation of one node (i,j,k): Eq. 7 where m > 0, gravity, tool
// contact with the closest tool (z-buffer merge; Eqs. 11, 15-19 with the
// friction clamped at zero tangential speed), then sticky walls.
__device__ __forceinline__ float3 grid_node_update(float m, float mvx, float mvy, float mvz, int i, int j, int k,
                                                   const DevParams &P, const ToolFrame *tools, int ntools) {
    if (!(m > 0.0f)) return make_float3(0.0f, 0.0f, 0.0f);
    float vx = mvx / m + P.dt * P.gx;
    float vy = mvy / m + P.dt * P.gy;
    float vz = mvz / m + P.dt * P.gz;
    if (ntools > 0) {
        const float xw = i * P.dx, yw = j * P.dx, zw = k * P.dx;
        float dmin, nbx, nby, nbz, pbx, pby, pbz;
        const int id = nearest_tool(xw, yw, zw, tools, ntools, dmin, nbx, nby, nbz, pbx, pby, pbz);
        if (id >= 0 && dmin < P.theta) {
            const ToolFrame &tf = tools[id];
            const float nx = tf.R[0] * nbx + tf.R[1] * nby + tf.R[2] * nbz;
            const float ny = tf.R[3] * nbx + tf.R[4] * nby + tf.R[5] * nbz;
            const float nz = tf.R[6] * nbx + tf.R[7] * nby + tf.R[8] * nbz;
            const float rx = xw - tf.T[0], ry = yw - tf.T[1], rz = zw - tf.T[2];
            const float cx = tf.u[0] + tf.w[1] * rz - tf.w[2] * ry;
            const float cy = tf.u[1] + tf.w[2] * rx - tf.w[0] * rz;
            const float cz = tf.u[2] + tf.w[0] * ry - tf.w[1] * rx;
            const float ux = vx - cx, uy = vy - cy, uz = vz - cz;      // Eq. 15
            const float vn = ux * nx + uy * ny + uz * nz;              // Eq. 16
            if (vn < 0.0f) {
                const float tx = ux - vn * nx, ty = uy - vn * ny, tz = uz - vn * nz;   // Eq. 17
                const float tn = sqrtf(tx * tx + ty * ty + tz * tz);
                float s = 0.0f;
                if (tn > 0.0f) s = fmaxf(tn + P.fric * vn, 0.0f) / tn;   // Eq. 18, clamped
                vx = s * tx + cx; vy = s * ty + cy; vz = s * tz + cz;    // Eq. 19
            }
        }
    }
    const int b = P.bound, hi = P.n - P.bound;
    if (i < b || j < b || k < b || i >= hi || j >= hi || k >= hi) vx = vy = vz = 0.0f;
    return make_float3(vx, vy, vz);
}

__device__ __forceinline__ bool finite3(float a, float b, float c) {
    return isfinite(a) && isfinite(b) && isfinite(c);
}

__device__ __forceinline__ void store_vc(const VCState &o, uint32_t s, float vx, float vy, float vz, const float C[9]) {
    o.vc0[s] = make_float4(vx, vy, vz, C[0]);
    o.vc1[s] = make_float4(C[1], C[2], C[3], C[4]);
    o.vc2[s] = make_float4(C[5], C[6], C[7], C[8]);
}

}  // namespace gbmpm
