/*
 * mpm.h -- C ABI of the GB300 MLS-MPM soft-tissue simulator.
 *
 * One handle owns one simulated scene: a set of Lagrangian particles of one
 * Neo-Hookean material on a fixed Eulerian grid covering the unit cube
 * [0,1)^3 (Sec. III-B: particles carry x, v, C, F; the grid carries mass and
 * momentum), plus up to MPM_MAX_TOOLS rigid collision shapes (Sec. III-C).
 * A sub-step is the paper's P2G (Eqs. 1-3, stress of Eqs. 5-6), grid
 * operation (Eq. 7, gravity, tool contact Eqs. 11-19, walls) and G2P with
 * advection (Eqs. 4, 8-10).  All numerical work runs in CUDA kernels for
 * sm_103a; this header exposes plain pointers and sizes only.
 *
 * Conventions shared by every entry point:
 *   - Every call returns an mpm_status.  On failure a description of the
 *     last error on the calling thread is available from mpm_last_error().
 *   - Device-side problems (non-finite values, inverted particles, particles
 *     leaving the grid, capacity overruns) set a sticky error word on the
 *     device.  Calls that synchronise (mpm_read_particles, mpm_synchronize,
 *     the introspection calls) report it; mpm_step reports it as soon as an
 *     earlier step that raised it has completed.  mpm_clear_error resets it.
 *   - Work is issued on the CUDA stream given at creation (or by
 *     mpm_set_stream) and is ordered with other work on that stream.
 *   - Layouts: positions and velocities are n x 3 row-major float arrays;
 *     F and C are n x 9 row-major (F[p*9 + 3*a + b] = F_ab of particle p).
 *     Particle p of every output is the particle loaded at index p.
 *   - Grid nodes are indexed [i][j][k], k fastest, node (i,j,k) at world
 *     position (i, j, k) * dx with dx = 1 / n_grid.
 *   - Caller-owned input buffers are copied; the caller may reuse them when
 *     the call returns.  The library owns every device buffer it allocates.
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef GBMPM_MPM_H
#define GBMPM_MPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpm_handle mpm_handle;

typedef enum mpm_status {
    MPM_OK = 0,
    MPM_ERR_ARG = -1,       /* invalid argument (NULL, out of range, wrong size) */
    MPM_ERR_ALLOC = -2,     /* device or host allocation failed */
    MPM_ERR_CUDA = -3,      /* a CUDA runtime call failed */
    MPM_ERR_NUMERIC = -4,   /* NaN/Inf in the state, or det F <= 0 (clamped to 1e-6 in ln) */
    MPM_ERR_DOMAIN = -5,    /* a particle's stencil left the grid (clamped to the grid) */
    MPM_ERR_TIMEOUT = -6,   /* a bounded device wait gave up */
    MPM_ERR_STATE = -7,     /* call not valid in the handle's current state */
    MPM_ERR_CAPACITY = -8,  /* an internal capacity was exceeded (see mpm_step) */
    MPM_ERR_CFL = -9        /* a particle moved more than one 4-cell block in a sub-step */
} mpm_status;

enum {
    MPM_MAX_TOOLS = 8,
    MPM_MAX_FIELDS = 16,      /* sampled distance fields per handle */
    MPM_MAX_FIELD_RES = 1024, /* samples per axis of one field */
    MPM_PIPELINE_FUSED = 0, /* block-sorted particles; one fused kernel per sub-step */
    MPM_PIPELINE_SPLIT = 1  /* unsorted particles; P2G, grid and G2P as separate kernels */
};

/* Tool shape kinds, shape[0] of mpm_set_tool_pose. */
enum { MPM_TOOL_NONE = -1, MPM_TOOL_CAPSULE = 0, MPM_TOOL_BOX = 1, MPM_TOOL_SAMPLED = 2 };

typedef struct mpm_config {
    int32_t n_grid;         /* nodes per axis: a power of two in [8, 512]; dx = 1/n_grid */
    int32_t bound;          /* sticky wall band in nodes, >= 0 (walls zero every velocity
                               component at nodes with an index < bound or >= n_grid - bound) */
    float dt;               /* sub-step Delta t in seconds, > 0 */
    float gravity[3];       /* m/s^2, added to grid velocities after Eq. 7 */
    float E;                /* Young's modulus (Pa), >= 0 */
    float nu;               /* Poisson's ratio, in [0, 0.5) */
    float rho;              /* density (kg/m^3), > 0; particle mass = rho * particle volume */
    float theta;            /* contact threshold: a node collides if its distance < theta */
    float friction_mu;      /* Coulomb coefficient of Eq. 18, >= 0 */
    int32_t pipeline;       /* MPM_PIPELINE_FUSED or MPM_PIPELINE_SPLIT */
    int32_t n_envs;         /* independent environments stepped together (0 or 1: one); more
                               than one needs the fused pipeline.  All share n_grid, dt,
                               gravity, bound, theta and friction_mu; each has its own particles,
                               material (mpm_set_env_material) and tools (mpm_set_env_tool_pose) */
    int64_t max_particles;  /* capacity of the handle over all environments, >= 1 */
} mpm_config;

/* Optional device allocator.  alloc returns a device pointer of at least
 * `bytes` bytes, 256-byte aligned, usable on `stream`, or NULL on failure;
 * free releases it.  With alloc == NULL the library uses cudaMalloc/cudaFree. */
typedef void *(*mpm_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*mpm_free_fn)(void *ptr, void *stream, void *ctx);

/* Create a handle for the current CUDA device.  cuda_stream: a cudaStream_t
 * (NULL = the legacy default stream).  Allocates every buffer sized by
 * cfg->max_particles and cfg->n_grid up front.  *out receives the handle. */
mpm_status mpm_create(const mpm_config *cfg, void *cuda_stream, mpm_alloc_fn alloc,
                      mpm_free_fn free_fn, void *ctx, mpm_handle **out);

/* Release every resource of the handle (waits for its stream first). */
mpm_status mpm_destroy(mpm_handle *h);

/* Replace the particle state with n particles (0 <= n <= max_particles).
 * x: n x 3 positions (required); v: n x 3 or NULL (zero); F: n x 9 or NULL
 * (identity); C: n x 9 or NULL (zero).  Handles with one environment only
 * (see mpm_load_batch).  particle_volume: V_p^0 (> 0), the
 * same for every particle (Table I).  on_device != 0: the pointers are device
 * memory readable on the handle's stream; otherwise host memory.  The stored
 * F is taken as already updated by Eq. 4, so the first P2G uses P(F) F^T of
 * the given F (Eq. 3).  Asynchronous for device inputs. */
mpm_status mpm_load_particles(mpm_handle *h, int64_t n, const float *x, const float *v,
                              const float *F, const float *C, float particle_volume,
                              int on_device);

/* Load every environment of a handle at once: counts[e] particles of
 * environment e (e < n_envs), stored one environment after the other in x,
 * v, F, C (layouts as for mpm_load_particles, NULL v/F/C as there);
 * particle_volumes[e] is V_p^0 of environment e.  counts and
 * particle_volumes are host arrays of n_envs entries.  Particle indices of
 * every output run over the environments in this order. */
mpm_status mpm_load_batch(mpm_handle *h, const int64_t *counts, const float *x, const float *v,
                          const float *F, const float *C, const float *particle_volumes,
                          int on_device);

/* Material of environment env: Young's modulus, Poisson's ratio (Eq. 6) and
 * density (mass = rho * particle volume).  Environments start with the
 * values of mpm_config.  A change applies from the next stress evaluation;
 * the grid already scattered keeps the previous values. */
mpm_status mpm_set_env_material(mpm_handle *h, int32_t env, float E, float nu, float rho);

/* mpm_set_tool_pose for environment env (mpm_set_tool_pose addresses
 * environment 0). */
mpm_status mpm_set_env_tool_pose(mpm_handle *h, int32_t env, int32_t tool_id, const double pose[6],
                                 const float shape[8]);

/* Set rigid tool tool_id (0 <= tool_id < MPM_MAX_TOOLS) (Sec. III-C).
 * pose: world translation T (3) then rotation vector (3): a reference-frame
 * point p sits at R p + T, R = exp([r]_x); grid nodes are mapped to the tool
 * frame by Eq. 11.  shape: 8 floats, shape[0] = kind; capsule: shape[1] =
 * radius, shape[2] = half-length of the axis segment along local y; box:
 * shape[1..3] = half extents; sampled: shape[1] = a field id returned by
 * mpm_add_sampled_field; kind MPM_TOOL_NONE removes the tool.  The pose
 * is the target for the end of the next mpm_step call: during that call the
 * tool moves uniformly (constant linear and angular velocity) from its
 * current pose to the target, and that rigid velocity is v_co of Eq. 15.
 * The first call for a tool places it without motion.  The pose is double
 * precision because the tool velocity is a difference of nearby poses.
 * Host arrays. */
mpm_status mpm_set_tool_pose(mpm_handle *h, int32_t tool_id, const double pose[6],
                             const float shape[8]);

/* Register a distance field precomputed in a tool's reference frame (the
 * offline SDF of Sec. III-C, Eqs. 12-14) for tools of kind MPM_TOOL_SAMPLED.
 * samples: res^3 floats, x fastest: samples[(k*res + j)*res + i] is the
 * signed distance at origin + spacing*(i, j, k) (reference frame, metres;
 * negative inside the tool).  The paper's field is res = 256 with
 * spacing = 1/256 and origin 0.  At a grid node with reference-frame position
 * x_ref the distance is the sample at floor((x_ref - origin)/spacing) on each
 * axis (Eq. 12) and the contact normal is the central difference of the
 * neighbouring samples (Eq. 14; one-sided at the faces of the field),
 * normalised; nodes outside the sampled volume are not in contact with the
 * tool.  res in [1, MPM_MAX_FIELD_RES]; at most MPM_MAX_FIELDS fields per
 * handle (MPM_ERR_CAPACITY beyond).  The samples are copied into device
 * memory owned by the handle (freed by mpm_destroy), so the caller's array
 * may be released on return; on_device != 0: samples is a device pointer,
 * otherwise a host array (checked for NaN).  Synchronises the stream.  Every
 * environment of the handle may use the field; *field_id receives its id
 * (0, 1, ... in registration order). */
mpm_status mpm_add_sampled_field(mpm_handle *h, int32_t res, const double origin[3], double spacing,
                                 const float *samples, int on_device, int32_t *field_id);

/* Advance n_substeps >= 0 sub-steps (P2G, grid operation, G2P; Sec. III-B).
 * Asynchronous on the handle's stream.  The fused pipeline folds a stable
 * counting sort of the particles by 4x4x4-cell grid block into each sub-step;
 * a block may receive particles from at most 512 source chunks of 256
 * particles per sub-step (MPM_ERR_CAPACITY otherwise). */
mpm_status mpm_step(mpm_handle *h, int32_t n_substeps);

/* mpm_read_particles without the wait, for streaming positions out while
 * the next sub-steps run: the state at this point of the handle's stream is
 * gathered on that stream into one of two device staging buffers, then
 * copied to the host arrays on a separate copy stream, overlapping the
 * sub-steps enqueued after it.  Host arrays (page-locked for the overlap),
 * any may be NULL.  The arrays of a call may be read once mpm_wait_read
 * (or a later call that waits) returns; a call waits on the GPU for the copy
 * two calls earlier before it refills that staging buffer. */
mpm_status mpm_read_particles_async(mpm_handle *h, float *x, float *v, float *F, float *C);

/* Wait for every copy mpm_read_particles_async started; returns the sticky
 * device status seen so far. */
mpm_status mpm_wait_read(mpm_handle *h);

/* Copy the particle state out in load order (n = the loaded count).  Any of
 * x (n x 3), v (n x 3), F (n x 9), C (n x 9) may be NULL to skip it.
 * on_device != 0: device pointers; otherwise host pointers.  Synchronises
 * the stream and returns the sticky device status. */
mpm_status mpm_read_particles(mpm_handle *h, float *x, float *v, float *F, float *C,
                              int on_device);

/* Thread-local description of the last failing call on this thread. */
const char *mpm_last_error(void);

/* ---------------------------------------------------------- introspection */

/* Number of loaded particles. */
mpm_status mpm_num_particles(mpm_handle *h, int64_t *n);

/* Sub-steps taken since the last load. */
mpm_status mpm_substeps_taken(mpm_handle *h, int64_t *count);

/* Wait for the handle's stream and return the sticky device status. */
mpm_status mpm_synchronize(mpm_handle *h);

/* Reset the sticky device error word. */
mpm_status mpm_clear_error(mpm_handle *h);

/* Use another stream for subsequent work (the caller orders the switch). */
mpm_status mpm_set_stream(mpm_handle *h, void *cuda_stream);

/* Grid mass and momentum that the next sub-step's grid operation starts from
 * (the P2G of the current particle state, Eqs. 1-2): n_envs x n_grid^3 x 4
 * floats (m, mv_x, mv_y, mv_z) per node, environment-major.  Synchronises. */
mpm_status mpm_read_grid(mpm_handle *h, float *grid, int on_device);

/* Grid velocities after the grid operation (Eq. 7, gravity, tools, walls)
 * applied to mpm_read_grid's state with the tool poses a following
 * mpm_step(h, 1) would use: n_envs x n_grid^3 x 3 floats.  Synchronises. */
mpm_status mpm_grid_velocity(mpm_handle *h, float *v, int on_device);

/* Fused pipeline only: the current order of the particles, i.e. the result
 * of the per-sub-step stable counting sort.  ids: n particle indices (load
 * order) sorted by grid-block key, ties in the order of the previous sort
 * (after a load: by particle index); keys: the block key of each entry,
 * bx + nb*(by + nb*bz) with nb = n_grid/4 and b = floor(x/dx - 0.5)/4
 * (clamped to the grid), plus e * nb^3 for a particle of environment e.
 * Host arrays of n entries.  Synchronises. */
mpm_status mpm_read_order(mpm_handle *h, uint32_t *ids, uint32_t *keys);

/* ------------------------------------------------------- surface extraction */

/* Iso-surface of environment env's tissue: the renderer's Marching Cubes
 * step of Sec. III, on the grid the next sub-step starts from.  The field
 * is the node density m_i / (rho dx^3) (about 1 inside the body, 0 outside);
 * the surface is density = iso, facing away from density >= iso.  Each grid
 * cell is split into six tetrahedra around its diagonal from its lowest to
 * its highest corner, each contributing 0, 1 or 2 triangles; the surface is
 * closed wherever it stays inside the grid.  Vertices are linear
 * interpolations on tetrahedron edges.  tri: up to max_tri triangles of 9
 * floats (three vertices x, y, z in metres), in cell order (i fastest, then
 * j, then k) and a fixed order inside a cell; *n_tri receives the total
 * (which may exceed max_tri: call again with a larger array).  on_device !=
 * 0: tri is a device pointer; otherwise a host array (the handle keeps a
 * device staging buffer).  Synchronises. */
mpm_status mpm_extract_surface(mpm_handle *h, int32_t env, float iso, float *tri, int64_t max_tri,
                               int64_t *n_tri, int on_device);

/* ------------------------------------------------------------ kernel tuning */

/* Configurations of the fused sub-step kernel: CTA size x passes of particles
 * staged per shared-memory P2G flush (x resident CTAs per SM).  More, smaller
 * CTAs waste fewer threads on sparsely filled grid blocks (small or batched
 * scenes); larger CTAs and groups amortise the per-block work on dense
 * blocks; two CTAs per SM with twice the registers shorten the latency chain
 * of a block when there are few blocks per CTA.  Not in the paper (its
 * Taichi kernels are tuned by Taichi); a utility of this library. */
enum {
    MPM_KERNEL_T256_G2 = 0, /* 256 threads, 512 particles per flush (the default) */
    MPM_KERNEL_T256_G1 = 1, /* 256 threads, 256 particles per flush */
    MPM_KERNEL_T128_G2 = 2, /* 128 threads, 256 particles per flush, particles copied 2 passes ahead */
    MPM_KERNEL_T128_G1 = 3, /* 128 threads, 128 particles per flush */
    MPM_KERNEL_T256_G2_C2 = 4, /* 256 threads, 512 particles per flush, 2 CTAs per SM, copied 2 passes ahead */
    MPM_KERNEL_CONFIGS = 5
};

/* Select the fused kernel configuration (fused pipeline; the split pipeline
 * ignores it).  MPM_ERR_ARG if out of range or not resident on this GPU. */
mpm_status mpm_set_kernel_config(mpm_handle *h, int32_t config);

/* The current configuration, its CTA size and the persistent grid size (CTAs
 * per launch); any output may be NULL. */
mpm_status mpm_get_kernel_config(mpm_handle *h, int32_t *config, int32_t *threads, int32_t *ctas);

/* Autotuner: time every configuration on the handle's own state (one
 * untimed call of n_substeps sub-steps, then three timed calls, each trial
 * starting from the same snapshot of the particles and tools), select the
 * one with the smallest median call time and restore the state as it was
 * (particle order inside the library may change; mpm_read_particles returns
 * the same values).  times_ms (MPM_KERNEL_CONFIGS floats: the median call
 * times, -1 for configurations that do not fit) and best may be NULL.  Needs a loaded fused-pipeline handle
 * (MPM_ERR_STATE).  Synchronises; allocates a snapshot of 24 floats per
 * particle, kept by the handle. */
mpm_status mpm_autotune(mpm_handle *h, int32_t n_substeps, float *times_ms, int32_t *best);

/* -------------------------------------------------- differentiable rollout */

/* Record a rollout of n_substeps sub-steps for mpm_tape_backward: sub-step k
 * moves every tool from its pose at the end of sub-step k-1 (for k = 0, its
 * current pose) to poses[(k * n_tools + t) * 6 ...] (T, rotation vector;
 * n_tools = highest tool slot in use + 1) -- the same as calling
 * mpm_set_tool_pose with those poses and mpm_step(1) n_substeps times.
 * The handle's state advances to the end of the rollout.  The particle state
 * is stored every checkpoint_every sub-steps (24 floats per particle each);
 * mpm_tape_backward recomputes the sub-steps in between.  The paper does not
 * differentiate its simulator (Sec. V names differentiable physics as future
 * work); this is the plain reverse mode of the sub-step defined above.
 * Needs a handle with one environment (MPM_ERR_STATE otherwise), on either
 * pipeline.  On MPM_PIPELINE_FUSED the last segment (the sub-steps after the
 * last checkpoint) is recorded as it runs, so mpm_tape_backward reverses it
 * without recomputing it.  poses: host array.  Device memory for the record is
 * taken from the handle's allocator and kept (and reused) until mpm_destroy. */
mpm_status mpm_tape_record(mpm_handle *h, int32_t n_substeps, const double *poses,
                           int32_t checkpoint_every);

/* Reverse mode of the recorded rollout.  x_bar (n x 3), v_bar (n x 3),
 * F_bar (n x 9), C_bar (n x 9): dL/d(final state) in load order; NULL = 0.
 * Outputs (each may be NULL): grad_material[2] = dL/dE, dL/dnu (through
 * Eq. 6); grad_poses = dL/dposes, laid out as mpm_tape_record's poses
 * (host, double); x0_bar, v0_bar, F0_bar, C0_bar = dL/d(state before the
 * rollout).  on_device applies to the float arrays (inputs and outputs);
 * grad_material and grad_poses are host arrays.  Each branch of the forward
 * pass (contact, approaching test, friction clamp, closest tool, walls,
 * m > 0) is held at the side taken; distances and sampled fields give no
 * derivative.  Material and tools must be unchanged since the record
 * (MPM_ERR_STATE).  Synchronises. */
mpm_status mpm_tape_backward(mpm_handle *h, const float *x_bar, const float *v_bar, const float *F_bar,
                             const float *C_bar, int on_device, double *grad_material, double *grad_poses,
                             float *x0_bar, float *v0_bar, float *F0_bar, float *C0_bar);

/* Inspection of a fused-pipeline record (for tests of the reverse mode): the
 * state sub-step c + j of the rollout started from, where c is the first
 * sub-step of the last segment (the last multiple of checkpoint_every below
 * n_substeps) and 0 <= j < n_substeps - c.  These are exactly the states the
 * reverse pass differentiates at, since it does not recompute that segment.
 * x (n x 3), v (n x 3), F (n x 9), C (n x 9) by load order; grid: the (m, mv)
 * grid that sub-step's grid operation read, n_grid^3 x 4 laid out as
 * mpm_read_grid lays it out (nodes outside the recorded blocks' regions hold
 * no mass and read as 0).  Any output may be NULL; on_device says where the
 * outputs live.  MPM_ERR_STATE without such a record: the split pipeline, no
 * mpm_tape_record, or an mpm_tape_backward since (it replays earlier segments
 * into the same buffers).  MPM_ERR_ARG for j out of range.  Synchronises. */
mpm_status mpm_tape_read_substep(mpm_handle *h, int32_t j, float *x, float *v, float *F, float *C, float *grid,
                                 int on_device);

/* ------------------------------------------------------ without allocation */

/* The stable block sort that mpm_load_particles performs, for callers that
 * must not allocate device memory: code running inside a host that owns all
 * of the GPU's memory through its own pool or a fixed budget, where a
 * cudaMalloc (or a framework allocator call) would fail or is not allowed.
 * The paper has no counterpart; this is a utility of this library.
 *
 * x: n x 3 particle positions in device memory.  ids, keys: device outputs of
 * n entries: the particle indices sorted by the block key of
 * floor(x/dx - 0.5) (dx = 1/n_grid, clamped to the grid), ties in index
 * order, and each entry's key bx + nb*(by + nb*bz), nb = n_grid/4 -- the same
 * result as mpm_read_order after mpm_load_particles.  n_grid: a power of two
 * in [8, 256]; n <= 2^30; larger sizes return MPM_ERR_ARG.
 *
 * Allocates nothing: its scratch is one static device array of about 3 MB
 * that every GPU using the library holds until the process exits.  Every
 * call looks up that array's address in the current context
 * (cudaGetSymbolAddress, with the device current), so a host driving the GPU
 * through its own context, or one that has reset the device, gets the right
 * copy; the first call in a context also loads the library's device code
 * there, so make that first call before any stream capture.  Every call
 * shares the array and leaves its contents behind (the counters are cleared
 * at the start of each call); calls that overlap on the GPU, on any streams,
 * race and must not be issued.  Runs on cuda_stream (NULL = legacy default)
 * and blocks the calling thread until that work is done; returns
 * MPM_ERR_NUMERIC / MPM_ERR_DOMAIN for non-finite or clamped positions (the
 * outputs then hold the order of the clamped keys, and the next call starts
 * clean). */
mpm_status mpm_block_sort_noalloc(const float *x, int64_t n, int32_t n_grid, uint32_t *ids,
                                  uint32_t *keys, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GBMPM_MPM_H */
