// launch.h -- host-side launchers of the library's kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gbmpm {

// capi.cu: the message mpm_last_error() returns on this thread
void set_last_error(const char *msg);

// kernels_split.cu
void launch_p2g_scatter(const DevParams &P, const PState &S, const VCState &V, uint32_t n, float4 *G, Ctrl *ctrl,
                        int grid, cudaStream_t st);
void launch_grid_update_dense(const DevParams &P, float4 *G, const ToolFrame *tools, int grid, cudaStream_t st);
// the grid operation of Gin (m, mv) into Gout (m, v)
void launch_grid_update_dense_to(const DevParams &P, const float4 *Gin, float4 *Gout, const ToolFrame *tools, int grid,
                                 cudaStream_t st);
void launch_g2p_split(const DevParams &P, const PState &S, const VCState &V, uint32_t n, const float4 *G, Ctrl *ctrl,
                      int grid, cudaStream_t st);
void launch_load_identity(const float *x, const float *v, const float *F, const float *C, uint32_t n, const PState &S,
                          const VCState &V, Ctrl *ctrl, int grid, cudaStream_t st);
void launch_read_out(const PState &S, const VCState &V, uint32_t n, float *x, float *v, float *F, float *C, int grid,
                     cudaStream_t st);
void launch_grid_to_dense(int n, int nb, int n_envs, const float4 *G, float4 *out, int grid, cudaStream_t st);
void launch_grid_velocity_dense(const DevParams &P, const float4 *G, const ToolFrame *tools, float *out, int grid,
                                cudaStream_t st);

// kernels_adjoint.cu: reverse mode of one split-pipeline sub-step.
// Adjoint of the particle state, row-major per particle (load order).
struct AdjState {
    float *x;   // n x 3
    float *v;   // n x 3
    float *C;   // n x 9
    float *F;   // n x 9
};
// Gv: grid after the forward grid operation (.yzw = velocity); Gb zeroed on
// entry, receives dL/d(grid velocity) in .yzw.  Vnext: v and C after the
// sub-step as the forward pass wrote them (same particle order as S), or
// null arrays to form them again from Gv.
void launch_adj_g2p(const DevParams &P, const PState &S, uint32_t n, const float4 *Gv, const AdjState &A, float4 *Gb,
                    const VCState &Vnext, int grid, cudaStream_t st);
// G: the (m, mv) grid the forward grid operation read; Gb in: velocity
// adjoint, out: (dL/dm, dL/dmv); tool_bar: ntools x 18 doubles accumulated.
// Optional block lists of 8 entries per recorded work-list block (a grid
// block, or kNoBlock), the number of those work-list blocks at *nlist: list,
// the only grid blocks that hold an adjoint; zlist, blocks whose nodes are
// cleared in zbuf.
constexpr uint32_t kNoBlock = 0xffffffffu;
struct AdjGridLists {
    const uint32_t *list = nullptr, *nlist = nullptr;
    const uint32_t *zlist = nullptr, *znlist = nullptr;
    float4 *zbuf = nullptr;
    // a byte range to bring into L2 for the next launch (the next reverse
    // sub-step's particle record), or none
    const void *prefetch = nullptr;
    size_t prefetch_bytes = 0;
};
void launch_adj_grid(const DevParams &P, const float4 *G, const ToolFrame *tools, float4 *Gb, double *tool_bar,
                     int grid, cudaStream_t st, const AdjGridLists &L = AdjGridLists());
void launch_adj_p2g(const DevParams &P, const PState &S, const VCState &V, uint32_t n, const float4 *Gb,
                    const AdjState &A, double *lame_bar, int grid, cudaStream_t st);

// kernels_reverse.cu: reverse mode of the fused sub-step over the blocks a
// recording sub-step listed (StepRecord, below).
struct StepRecord;
struct ReverseArgs;
// CTAs per SM of the reverse sub-step (also opts it into its shared memory)
int reverse_step_ctas_per_sm();
// do_p2g && do_g2p: reverse of G2P of sub-step k and P2G of sub-step k+1;
// do_g2p alone: the last sub-step of a rollout; do_p2g alone: the reverse of
// the first sub-step's P2G at the initial state.  dependent: launched as a
// programmatic dependent of the stream's previous kernel (which then must be
// the only work it depends on: its set-up reads the record before waiting).
void launch_reverse_step(bool do_p2g, bool do_g2p, const DevParams &P, const ReverseArgs &R, int grid,
                         cudaStream_t st, bool dependent);

// kernels_surface.cu: iso-surface of the grid density m / (rho dx^3) of
// environment env.  counts: (n-1)^3 + 1 entries, left holding the exclusive
// prefix of the per-cell triangle counts (last entry: the total); sums:
// ceil(((n-1)^3 + 1) / 1024) + 1 entries.
void launch_surface_count_scan(const float4 *G, int n, int nb, uint32_t nbe, uint32_t env, float scale, float iso,
                               uint32_t *counts, uint32_t *sums, int grid, cudaStream_t st);
// triangles (9 floats each) in cell order, the first max_tri of them
void launch_surface_emit(const float4 *G, int n, int nb, uint32_t nbe, uint32_t env, float scale, float iso, float dx,
                         const uint32_t *offsets, float *tri, uint64_t max_tri, int grid, cudaStream_t st);

// kernels_sort.cu: stable counting sort of particles by grid block at load.
struct SortScratch {
    uint32_t *keys;     // n
    uint32_t *counts;   // nblocks
    uint32_t *offsets;  // nblocks + 1
    uint32_t *cursor;   // nblocks
    uint32_t *perm;     // n: slot -> particle index
};
// counts/offsets/perm of the stable counting sort of particles by the block
// of floor(x/dx - 0.5) (x: n x 3 row-major, device).  counts must be zero on
// entry.  keys holds the per-particle keys during the sort and is left as
// scratch (overwritten where a block holds more than 2,048 particles).
void launch_block_sort(const DevParams &P, const float *x, uint32_t n, const SortScratch &s, Ctrl *ctrl, int grid,
                       cudaStream_t st);
// Place particle perm[j] in slot j and build the run tables of sub-step
// `step` (one chunk per non-empty block, index = block id).
struct FusedBufs;
void launch_place_sorted(const DevParams &P, const float *x, const float *v, const float *F, const float *C,
                         uint32_t n, const SortScratch &s, const PState &S, const VCState &V, int grid,
                         cudaStream_t st);
void launch_init_tables(const DevParams &P, const SortScratch &s, const FusedBufs &B, uint32_t step, int grid,
                        cudaStream_t st);

// kernel_fused.cu
struct FusedBufs {
    PState P[2];
    VCState vc;               // v and C of the last sub-step of a call, slot-aligned with P[current]
    Chunk *chunks[2];
    BlockTab *tabs[2];
    uint32_t *alist[2];       // active blocks by sub-step parity
    uint32_t *clist[3];       // grid blocks to clear, by sub-step mod 3
    float4 *G[3];             // grid buffers by sub-step mod 3
    uint4 *inbox[2];          // per destination block: kInbox entries (first slot, count, stamp, 0)
    uint32_t *astamp;         // per block: last sub-step it was put on an active list
    uint32_t *gstamp;         // per block: last sub-step it was put on a clear list
    Ctrl *ctrl;
    uint32_t nblocks;
};
// What a recording fused sub-step writes for the reverse mode (all device
// arrays): each block's input particles in block-contiguous order (n
// entries), per block its (first, count) range, the blocks in work order and
// their number.
// Particles are recorded at their output position of the sub-step (inside
// their block's output range), so that the reverse pass reads the adjoint the
// later reverse sub-step left at that position with coalesced loads.
struct StepRecord {
    float4 *xi, *f0, *f1;
    float *f2;
    uint32_t *src;       // each particle's position in the sub-step's input arrays
    uint2 *blk;          // nblocks: the particle range of the block at each work-list index
    uint32_t *act;       // nblocks
    uint32_t *nact;      // 1
    float4 *grid;        // the grid the sub-step read, over the 6^3 region of every listed block (node layout)
    float4 *vgrid;       // the grid velocities after the grid operation (.xyz), over the same regions
    VCState vc;          // each particle's v and C after the sub-step (n entries, same order as xi)
};
// Inputs and outputs of one reverse sub-step (kernels_reverse.cu).
struct ReverseArgs {
    StepRecord rec;            // sub-step k's input particles by block
    const float4 *gbar_next;   // dL/d(m, mv) of G_{k+1} (do_p2g)
    float4 *vbar;              // dL/dV_k in .yzw, accumulated (do_g2p)
    AdjState lam;              // particle adjoints by particle id
    // Between the sub-steps of a segment the adjoint of a state is (x, F) only
    // (G2P does not read v and C, and P2G's part of them stays in the thread),
    // kept by position as three float4 per particle: (xb, Fb0), Fb1..4, Fb5..8
    // at [p], [np + p], [2 np + p].  lam_in_by_id: read this sub-step's
    // incoming adjoint from lam (the segment's last sub-step); otherwise from
    // lp_in at the particle's recorded (output) position.  lam_out_by_id:
    // write the outgoing one to lam (the segment's first sub-step); otherwise
    // to lp_out at the particle's input position (rec.src).
    const float4 *lp_in;
    float4 *lp_out;
    uint32_t np;
    int lam_in_by_id, lam_out_by_id;
    const float *v0, *C0;      // initial v (n x 3), C (n x 9) by id (do_p2g alone)
    double *lame_part;         // per CTA: its part of dL/dmu, dL/dlambda, accumulated
    // (do_g2p) the grid blocks the sub-step scatters into -- every recorded block
    // b and b + {0,1}^3 -- listed once in touch_list (8 entries per work-list
    // block, kNoBlock where a block is out of the grid or listed by another),
    // marked in stamp with value sv
    uint32_t *stamp, sv, *touch_list;
    uint32_t *touch_n;         // receives the number of work-list blocks (do_g2p)
};
// config (MPM_KERNEL_*): 0 = 256 threads, 2 passes per P2G flush; 1 = 256, 1;
// 2 = 128, 2; 3 = 128, 1; 4 = 256, 2 with 2 CTAs per SM.  Configurations 2 and
// 4 copy each pass's particles two passes ahead, the others one pass ahead.
void launch_fused_step(const DevParams &P, const FusedBufs &B, const ToolFrame *tools, bool write_vc, int grid,
                       int config, cudaStream_t st);
int fused_step_occupancy(int config);
int fused_step_threads(int config);
int fused_record_occupancy();
void launch_fused_step_record(const DevParams &P, const FusedBufs &B, const ToolFrame *tools, const StepRecord &rec,
                              int grid, cudaStream_t st);
constexpr int kFusedConfigs = 5;
constexpr int kFusedMinThreads = 128;     // chunk tables are sized for the smallest CTA
// Inbox of a block: entry d * kNpMax + p holds the run of source pass p
// coming from direction d (source block = block - dir(d)); the last entry,
// stamped, says that some source had more than kNpMax passes.
constexpr int kNpMax = 4;
constexpr int kInbox = 27 * kNpMax + 1;

}  // namespace gbmpm
