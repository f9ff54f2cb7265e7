// kernel_fused.cu -- one MLS-MPM sub-step as a single persistent kernel over
// the occupied 4x4x4-cell grid blocks.
//
// Sub-step k reads the grid G_k (mass, momentum after P2G of the particles at
// x_k) and the particles, grouped by the block of their stencil base, and
// writes x_{k+1}, F_{k+1} and the P2G of the new state into G_{k+1}:
//
//   per occupied block b (one CTA iteration):
//   1. grid operation (Eq. 7, gravity, tool contact Eqs. 11, 15-19, walls) of
//      the 6^3 nodes that the stencils of b's particles touch, into shared
//      memory;
//   2. per particle (passes of one particle per thread): G2P (Eqs. 8-9), F
//      update (Eq. 4), advection (Eq. 10), Kirchhoff stress of the new F
//      (Eqs. 5-6) and the affine momentum A = m C - dt V^0 (4/dx^2) tau;
//   3. a stable counting sort of the particles by their new block: every pass
//      writes its particles grouped by the direction (-1..1)^3 to their new
//      block and records where each group starts; the next sub-step's CTA for
//      block b' reads the runs heading to b' from its 27 neighbours, in
//      ascending source-block order;
//   4. P2G (Eqs. 1-3) of up to 2 passes of new particle states at a time into an
//      8^3-node shared arena around b.  The arena accumulates in 32-bit fixed
//      point with native shared integer atomics (shared float atomics are
//      several times slower): mass in units of m_p 2^-22, momentum in units of
//      B 2^-22 where B bounds every contribution of the group, so no
//      contribution exceeds 2^22 and no node sum of <= 512 particles can
//      overflow; the integer sums are exact, hence independent of the order of
//      the atomics.  A particle that moved further than one cell scatters
//      straight into G_{k+1} with float atomics instead.
//   5. the arena is converted back to floats and added to G_{k+1} with float4
//      atomics (only the 6^3 nodes around b when every base cell lies in b),
//      and the nodes read are returned to zero.
//
// G2P and P2G run their x/y (and z/mass) components on the packed f32x2 pipe.
//
// Grid buffers rotate over three slots (read G_k, write G_{k+1}, clear
// G_{k-1} for reuse), particle buffers and run tables over two; the last CTA
// to finish resets the per-launch counters and advances the sub-step index.
#include "common.cuh"
#include "launch.h"

namespace gbmpm {

namespace {

constexpr int CMAX = 512;      // run candidates (source chunk x direction) per block
constexpr float kFix = 4194304.0f;      // 2^22
constexpr float kMagic = 12582912.0f;   // 1.5 * 2^23: float -> nearest int for |v| < 2^22
// arena node (x, y, z) in [0,8)^3 sits at x + kAy y + kAz z: kAz = 68 keeps the
// bases of a z-pair of cells in distinct shared-memory banks
constexpr int kAy = 8, kAz = 68, kArena = 8 * kAz;

// Shared memory of a CTA of T threads that stages GP passes (GP T particles)
// per arena flush.
// PD: particle copies in flight per thread (a pass's particle is copied PD
// passes ahead of its use)
template <int T, int GP, int PD = 1>
struct FusedSmem {
    static constexpr int NW = T / 32;
    static constexpr int GROUP = GP * T;
    // double-buffered per-block inputs, prefetched with cp.async one block ahead:
    // the 6^3 grid nodes [4b, 4b+5]^3 (mass, momentum; turned into velocities
    // in place by the grid operation) and the block's inbox of incoming runs
    float4 graw[2][216];
    uint4 inbox[2][kInbox];
    EnvParams ep[2];               // the block's environment: material
    ToolFrame tools[2][kMaxTools]; // and its tool frames for this sub-step
    uint32_t items[2], bids[2];
    int acc[4][kArena];            // P2G arena over nodes [4b-1, 4b+6]^3 (fixed point, padded strides)
    // staged P2G inputs of one group: packed arena base, fx (3), q (3), A dx (9)
    int st_base[GROUP];
    // the group's particles bucketed by the shared-memory bank of their arena
    // base: rank within the bucket (and the bucket) per slot, bucket sizes, and
    // the slots in bucket order
    uint16_t st_key[GROUP];
    uint16_t order[GROUP];
    uint32_t ccount[32];
    float st_f[3][GROUP];
    float st_q[3][GROUP];
    float st_a[9][GROUP];
    // each thread's particle of the current pass, prefetched with cp.async a pass
    // ahead (a thread reads and refills only its own slot)
    float4 pxi[PD][T], pf0[PD][T], pf1[PD][T];
    float pf2[PD][T];
    uint32_t cand_start[CMAX];     // first slot of each run
    uint32_t cand_pre[CMAX + 1];   // exclusive prefix of run lengths
    uint32_t lane_first[27], lane_off[27];
    // per pass parity: per direction, each warp's count of it (one byte per
    // warp, so that a lane sums all warps' counts of its direction in one load)
    static constexpr int NWP = NW <= 4 ? 4 : 8;
    alignas(8) uint8_t wcnt[2][28][NWP];
    uint32_t ncand, total, out_base, chunk_first, npass, mask, bmax, wide;
};

// resident CTAs per SM for which a configuration is compiled: 228 KB of shared
// memory per SM with 1 KB reserved per CTA, 64 K registers
template <int T, int GP>
constexpr int kMinBlocks = T == 256 ? 3 : (GP == 1 ? 5 : 4);
static_assert(3 * (sizeof(FusedSmem<256, 2>) + 1024) <= 228 * 1024, "shared memory for three CTAs per SM");
static_assert(4 * (sizeof(FusedSmem<128, 2>) + 1024) <= 228 * 1024, "shared memory for four CTAs per SM");
static_assert(5 * (sizeof(FusedSmem<128, 1>) + 1024) <= 228 * 1024, "shared memory for five CTAs per SM");
static_assert(4 * (sizeof(FusedSmem<128, 2, 2>) + 1024) <= 228 * 1024, "configuration 2: four CTAs per SM");
static_assert(2 * (sizeof(FusedSmem<256, 2, 2>) + 1024) <= 228 * 1024, "configuration 4: two CTAs per SM");

__device__ __forceinline__ int dir_dx(int d) { return d % 3 - 1; }
__device__ __forceinline__ int dir_dy(int d) { return (d / 3) % 3 - 1; }
__device__ __forceinline__ int dir_dz(int d) { return d / 9 - 1; }

__device__ __forceinline__ void mark_clear(const FusedBufs &B, uint32_t g, uint32_t stamp, int slot) {
    if (atomicExch(&B.gstamp[g], stamp) != stamp) B.clist[slot][atomicAdd(&B.ctrl->nclear[slot], 1u)] = g;
}

// nearest integer of v (|v| < 2^22) via the float mantissa
__device__ __forceinline__ int fix_round(float scaled_plus_magic) {
    return __float_as_int(scaled_plus_magic) - 0x4B400000;
}

// G[addr] += v as one vector reduction (no value returned)
__device__ __forceinline__ void red_add4(float4 *addr, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    const int bytes = valid ? 16 : 0;   // 0: fill with zeros, read nothing
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gmem), "r"(bytes) : "memory");
}
// 16 bytes into shared memory without allocating in L1 (streamed particle state)
__device__ __forceinline__ void cp_async16_cg(void *smem, const void *gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_but_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_but_two() { asm volatile("cp.async.wait_group 2;\n" ::: "memory"); }

// Slot of logical index j among the block's incoming runs (binary search of
// the runs' exclusive prefix).
template <class Smem>
__device__ __forceinline__ uint32_t source_slot(const Smem &s, uint32_t ncand, uint32_t j) {
    int lo = 0, hi = (int)ncand - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s.cand_pre[mid] <= j) lo = mid; else hi = mid - 1;
    }
    return s.cand_start[lo] + (j - s.cand_pre[lo]);
}

// Start copying the particle with logical index j into this thread's slot.
template <class Smem>
__device__ __forceinline__ void prefetch_particle(Smem &s, const PState &in, uint32_t ncand, uint32_t j, int tid,
                                                  int set) {
    const uint32_t src = source_slot(s, ncand, j);
    cp_async16_cg(&s.pxi[set][tid], &in.xi[src]);
    cp_async16_cg(&s.pf0[set][tid], &in.f0[src]);
    cp_async16_cg(&s.pf1[set][tid], &in.f1[src]);
    cp_async4(&s.pf2[set][tid], &in.f2[src]);
}

// Start copying global block b's grid region of G_k, its inbox, and its
// environment's material and tool frames into buffer buf.
template <int T, class Smem>
__device__ __forceinline__ void prefetch_block(Smem &s, int buf, uint32_t b, const uint4 *__restrict__ inbox_in,
                                               const float4 *__restrict__ Gcur, const DevParams &P,
                                               const ToolFrame *__restrict__ tools, int tid) {
    const uint32_t e = b / P.nbe, bl = b % P.nbe;
    const int nb = P.nb, n = P.n;
    const int bx = bl % nb, by = (bl / nb) % nb, bz = bl / (nb * nb);
    constexpr int kTw = (int)(sizeof(ToolFrame) / 16);   // 16-byte words per frame
    const int ntw = P.tstride * kTw;
    for (int q = tid; q < 216 + kInbox + 2 + ntw; q += T) {
        if (q < 216) {
            const int i = 4 * bx + q % 6, j = 4 * by + (q / 6) % 6, k = 4 * bz + q / 36;
            const bool ok = i < n && j < n && k < n;
            cp_async16(&s.graw[buf][q], ok ? (const void *)&Gcur[node_addr_env(e, i, j, k, nb, P.nbe)] : (const void *)Gcur,
                       ok);
        } else if (q < 216 + kInbox) {
            const int x = q - 216;
            cp_async16(&s.inbox[buf][x], &inbox_in[(size_t)b * kInbox + x], true);
        } else if (q < 216 + kInbox + 2) {
            const int x = q - 216 - kInbox;
            cp_async16(reinterpret_cast<uint4 *>(&s.ep[buf]) + x, reinterpret_cast<const uint4 *>(&P.envp[e]) + x, true);
        } else {
            const int x = q - 216 - kInbox - 2;
            cp_async16(reinterpret_cast<uint4 *>(&s.tools[buf][0]) + x,
                       reinterpret_cast<const uint4 *>(tools + (size_t)e * P.tstride) + x, true);
        }
    }
    cp_async_commit();
}


// MINB: resident CTAs per SM the configuration is compiled for (the register budget)
// RECORD: also write, for the reverse mode, every block's input particles at
// their output positions (inside the range [out_base, out_base + total) the
// block's output was allocated) with their input positions, the list of
// blocks in work order with each one's range, the list's length, and the grid
// of each block's region before and after the grid operation.
template <bool WRITE_VC, int T, int GP, int MINB = kMinBlocks<T, GP>, bool RECORD = false, int PD = 1>
__global__ void __launch_bounds__(T, MINB) k_fused_step(DevParams P, FusedBufs B,
                                                                     const ToolFrame *__restrict__ tools,
                                                                     StepRecord rec) {
    using Smem = FusedSmem<T, GP, PD>;
    static_assert(PD == 1 || PD == 2, "one or two particle copies in flight");
    constexpr int NW = Smem::NW, GROUP = Smem::GROUP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &s = *reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Ctrl *ctrl = B.ctrl;
    const uint32_t step = *(volatile uint32_t *)&ctrl->step;
    const int par = step & 1, m3 = step % 3;
    const int m3n = (m3 + 1) % 3, m3c = (m3 + 2) % 3;
    const PState in = par ? B.P[1] : B.P[0];
    const PState out = par ? B.P[0] : B.P[1];
    const Chunk *__restrict__ cin = par ? B.chunks[1] : B.chunks[0];
    Chunk *__restrict__ cout = par ? B.chunks[0] : B.chunks[1];
    const BlockTab *__restrict__ tin = par ? B.tabs[1] : B.tabs[0];
    BlockTab *__restrict__ tout = par ? B.tabs[0] : B.tabs[1];
    const float4 *__restrict__ Gcur = B.G[m3];
    float4 *Gnext = B.G[m3n];
    float4 *Gclr = B.G[m3c];
    const uint4 *__restrict__ inbox_in = par ? B.inbox[1] : B.inbox[0];
    uint4 *__restrict__ inbox_out = par ? B.inbox[0] : B.inbox[1];
    const uint32_t *__restrict__ act = B.alist[par];
    uint32_t *act_next = B.alist[par ^ 1];
    // the active blocks: heavy ones listed from the front, light ones from the
    // back, and handed out heavy first so that the launch ends on short items
    const unsigned long long nhl = *(volatile unsigned long long *)&ctrl->nactive[par][0];
    const uint32_t nheavy = (uint32_t)nhl, nact = (uint32_t)nhl + (uint32_t)(nhl >> 32);
    const uint32_t acap = B.nblocks;
    auto item_block = [&](uint32_t it) -> uint32_t {
        return it >= nact ? 0u : (it < nheavy ? act[it] : act[acap - 1u - (it - nheavy)]);
    };
    const uint32_t nclr = *(volatile uint32_t *)&ctrl->nclear[m3c];
    const uint32_t *__restrict__ clr = B.clist[m3c];
    const uint32_t nparticles = ctrl->n_particles;
    const uint32_t nchunk_cap = B.nblocks + nparticles / T + 1;
    const int nb = P.nb, n = P.n;
    const uint32_t nbe = P.nbe;
    uint32_t err = 0;

    // prologue: work item blockIdx.x first (the shared counter hands out items
    // gridDim.x, gridDim.x + 1, ... afterwards) and its inputs
    if (tid == T - 1) {
        const uint32_t it = blockIdx.x;
        s.items[0] = it;
        s.bids[0] = item_block(it);
    }
    __syncthreads();
    if (s.items[0] < nact) prefetch_block<T>(s, 0, s.bids[0], inbox_in, Gcur, P, tools, tid);
    // the P2G arena starts at zero; every flush returns the nodes it read to zero
    for (int q = tid; q < 4 * kArena; q += T) (&s.acc[0][0])[q] = 0;
    // 0. while the first block's inputs land: clear the grid blocks G_{k-1} touched,
    //    so that sub-step k+1 can scatter into it (a different buffer from G_k)
    for (uint32_t q = blockIdx.x * T + tid; q < nclr * 64u; q += gridDim.x * T)
        Gclr[clr[q >> 6] * 64u + (q & 63u)] = make_float4(0.f, 0.f, 0.f, 0.f);
    cp_async_wait_all();
    __syncthreads();

    for (int cb = 0;; cb ^= 1) {
        const uint32_t item = s.items[cb];
        if (item >= nact) break;
        const uint32_t b = s.bids[cb];                 // global block
        if (RECORD && tid == 0) rec.act[item] = b;
        const uint32_t env = b / nbe, bl = b % nbe;     // environment, block inside it
        const uint32_t eb0 = env * nbe;                 // first global block of the environment
        const int bx = bl % nb, by = (bl / nb) % nb, bz = bl / (nb * nb);
        const EnvParams &ep = s.ep[cb];
        const float m = ep.mass;
        // the next work item: the atomic is issued here and its result is
        // consumed after this thread's share of the grid operation
        uint32_t next_item = 0;
        if (tid == T - 1) next_item = gridDim.x + atomicAdd(&ctrl->work, 1u);
        uint32_t alloc_ob = 0, alloc_cf = 0;     // thread 0: the block's output range and chunks
        float4 *gv = s.graw[cb];

        // 1. grid operation of the 6^3 G2P region, in place (warps 1 ..)
        for (int q = tid - 32; q >= 0 && q < 216; q += T - 32) {
            const int i = 4 * bx + q % 6, j = 4 * by + (q / 6) % 6, k = 4 * bz + q / 36;
            const float4 g = gv[q];
            float3 v = make_float3(0.f, 0.f, 0.f);
            if (i < n && j < n && k < n) v = grid_node_update(g.x, g.y, g.z, g.w, i, j, k, P, s.tools[cb], ep.ntools);
            gv[q] = make_float4(v.x, v.y, v.z, 0.f);
            if (RECORD && i < n && j < n && k < n) {
                const uint32_t a = node_addr_env(env, i, j, k, nb, nbe);
                rec.grid[a] = g;
                rec.vgrid[a] = make_float4(v.x, v.y, v.z, 0.f);
            }
        }
        if (tid < 32) s.ccount[tid] = 0u;
        for (int q = tid; q < 2 * 28 * Smem::NWP / 4; q += T) reinterpret_cast<uint32_t *>(&s.wcnt[0][0][0])[q] = 0u;
        if (tid == T - 1) {
            s.items[cb ^ 1] = next_item;
            s.bids[cb ^ 1] = item_block(next_item);
        }
        // 2. warp 0: the runs heading to b, in ascending source-block order
        //    (direction d = 26 .. 0, source pass 0 .. 3), with their exclusive
        //    prefix = logical index of each run's first particle
        if (warp == 0) {
            const uint4 *ib = s.inbox[cb];
            uint32_t nc = 0, carry = 0;
            if (ib[kInbox - 1].x != step) {
                for (int base = 0; base < 27 * kNpMax; base += 32) {
                    const int idx = base + lane;
                    uint4 e = make_uint4(0u, 0u, 0u, 0u);
                    if (idx < 27 * kNpMax) e = ib[(26 - (idx / kNpMax)) * kNpMax + (idx % kNpMax)];
                    const bool ok = idx < 27 * kNpMax && e.z == step && e.y > 0u;
                    const unsigned bal = __ballot_sync(0xffffffffu, ok);
                    const uint32_t cnt = ok ? e.y : 0u;
                    uint32_t incl = cnt;
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += y;
                    }
                    if (ok) {
                        const uint32_t pos = nc + __popc(bal & ((1u << lane) - 1u));
                        s.cand_start[pos] = e.x;
                        s.cand_pre[pos] = carry + incl - cnt;
                    }
                    nc += __popc(bal);
                    carry += __shfl_sync(0xffffffffu, incl, 31);
                }
            } else {
                // a source wrote more passes than the inbox holds: walk its run tables
                uint32_t np = 0, first = 0;
                if (lane < 27) {
                    const int d = 26 - lane;
                    const int sx = bx - dir_dx(d), sy = by - dir_dy(d), sz = bz - dir_dz(d);
                    if (sx >= 0 && sy >= 0 && sz >= 0 && sx < nb && sy < nb && sz < nb) {
                        const BlockTab t = tin[eb0 + block_id(sx, sy, sz, nb)];
                        if (t.stamp == step) { np = t.npass; first = t.first; }
                    }
                }
                uint32_t incl = np;
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (lane < 27) { s.lane_first[lane] = first; s.lane_off[lane] = incl - np; }
                uint32_t ncand = __shfl_sync(0xffffffffu, incl, 26);
                if (ncand > CMAX) { ncand = CMAX; err |= kErrCapacity; }
                __syncwarp();
                for (uint32_t c0 = 0; c0 < ncand; c0 += 32) {
                    const uint32_t c = c0 + lane;
                    uint2 r = make_uint2(0u, 0u);
                    if (c < ncand) {
                        int l = 0;
                        while (l < 26 && s.lane_off[l + 1] <= c) ++l;
                        r = cin[s.lane_first[l] + (c - s.lane_off[l])].run[26 - l];
                    }
                    uint32_t incl2 = r.y;
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, incl2, o);
                        if (lane >= o) incl2 += y;
                    }
                    if (c < ncand) { s.cand_start[c] = r.x; s.cand_pre[c] = carry + incl2 - r.y; }
                    carry += __shfl_sync(0xffffffffu, incl2, 31);
                }
                nc = ncand;
            }
            __syncwarp();
            if (lane == 0) {
                s.ncand = nc;
                s.cand_pre[nc] = carry;
                s.total = carry;
                s.npass = (carry + T - 1) / T;
                // issued here, consumed after the barrier below
                alloc_ob = atomicAdd(&ctrl->part_alloc, carry);
                alloc_cf = atomicAdd(&ctrl->chunk_alloc, (carry + T - 1) / T);
                s.mask = 0;
                s.bmax = 0;
                s.wide = 0;
            }
        }
        __syncthreads();
        const uint32_t ncand = s.ncand;
        const uint32_t total = s.total, npass = s.npass;
        // thread 0: the block's table for the next sub-step and its output range,
        // read by every thread after the first pass's barrier; if the allocation
        // overflowed, the range starts past the end of the particle and chunk
        // arrays and nothing is written
        if (tid == 0) {
            BlockTab t;
            t.pad = 0;
            const bool fit = alloc_ob + total <= nparticles && alloc_cf + npass <= nchunk_cap;
            if (fit) {
                t.stamp = step + 1; t.first = alloc_cf; t.npass = npass;
            } else {
                err |= kErrCapacity;
                t.stamp = 0; t.first = 0; t.npass = 0;
            }
            tout[b] = t;
            if (RECORD) rec.blk[item] = make_uint2(fit ? alloc_ob : 0u, fit ? total : 0u);
            s.out_base = fit ? alloc_ob : nparticles;
            s.chunk_first = fit ? alloc_cf : nchunk_cap;
        }
        // this thread's particle of the first pass, then the next block's inputs;
        // both land while this block computes
        if (npass > 0 && (uint32_t)tid < total) prefetch_particle(s, in, ncand, (uint32_t)tid, tid, 0);
        cp_async_commit();
        if (PD == 2) {   // and the second pass's
            if (npass > 1 && (uint32_t)(T + tid) < total) prefetch_particle(s, in, ncand, (uint32_t)(T + tid), tid, 1);
            cp_async_commit();
        }
        if (s.items[cb ^ 1] < nact) prefetch_block<T>(s, cb ^ 1, s.bids[cb ^ 1], inbox_in, Gcur, P, tools, tid);
        else cp_async_commit();
        const int ox = 4 * bx - 1, oy = 4 * by - 1, oz = 4 * bz - 1;   // arena origin

        for (uint32_t pass = 0; pass < npass; ++pass) {
            const uint32_t j = pass * T + tid;
            const bool valid = j < total;
            const int slot = (pass % GP) * T + tid;    // staging slot within the group
            int d = 31;
            float nxp = 0.f, nyp = 0.f, nzp = 0.f, idf = 0.f, Fn[9], Cm[9], vx = 0.f, vy = 0.f, vz = 0.f;
            // this pass's particle is in the slot; the next block's inputs may still be landing
            // every thread commits, in order: pass 0's particle, [PD = 2: pass 1's
            // particle,] the next block's inputs, then one group per pass holding
            // the particle of pass + PD.  Wait for this pass's particle only.
            if (PD == 1) {
                if (pass == 0) cp_async_wait_but_one(); else cp_async_wait_all();
            } else {
                if (pass <= 1) cp_async_wait_but_two(); else cp_async_wait_but_one();
            }
            float4 xi = make_float4(0.f, 0.f, 0.f, 0.f), a0 = xi, a1 = xi;
            float f2 = 0.f;
            const int ps = (int)(pass % PD);   // slot set of this pass's particle
            if (valid) { xi = s.pxi[ps][tid]; a0 = s.pf0[ps][tid]; a1 = s.pf1[ps][tid]; f2 = s.pf2[ps][tid]; }
            const uint32_t jn = j + PD * T;
            if (valid) {
                const float F[9] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, f2};
                idf = xi.w;
                // --- G2P from the shared velocities (Eqs. 8-9)
                int gx, gy, gz;
                const float fx = stencil_axis(xi.x, P.inv_dx, n, gx, err);
                const float fy = stencil_axis(xi.y, P.inv_dx, n, gy, err);
                const float fz = stencil_axis(xi.z, P.inv_dx, n, gz, err);
                int lx = gx - 4 * bx, ly = gy - 4 * by, lz = gz - 4 * bz;
                if (lx < 0 || lx > 3 || ly < 0 || ly > 3 || lz < 0 || lz > 3) {
                    err |= kErrCfl;
                    lx = min(max(lx, 0), 3); ly = min(max(ly, 0), 3); lz = min(max(lz, 0), 3);
                }
                float wx[3], wy[3], wz[3];
                bspline_weights(fx, wx);
                bspline_weights(fy, wy);
                bspline_weights(fz, wz);
                // With the stencil offset o = (ii, jj, kk) - f (cell units), the
                // affine sum of Eq. 9 is sum w v o^T = sum w v (ii, jj, kk)^T - v f^T:
                // the moments about the stencil base need no per-node offset and
                // vanish on the ii = 0 (jj = 0, kk = 0) layers.  The x and y
                // components run on the packed f32x2 pipe.
                const float2 w0 = make_float2(wx[0], wx[0]), w1 = make_float2(wx[1], wx[1]);
                const float2 w2 = make_float2(wx[2], wx[2]), w2d = make_float2(2.f * wx[2], 2.f * wx[2]);
                float2 vxy = make_float2(0.f, 0.f), mxy = vxy, myy = vxy, mzy = vxy;   // v, and moments along x, y, z
                float vzz = 0.f, mxz = 0.f, myz = 0.f, mzz = 0.f;
#pragma unroll
                for (int kk = 0; kk < 3; ++kk) {
#pragma unroll
                    for (int jj = 0; jj < 3; ++jj) {
                        const float wjk = wy[jj] * wz[kk];
                        const float2 wjk2 = make_float2(wjk, wjk);
                        const float4 *row = &gv[lx + 6 * (ly + jj) + 36 * (lz + kk)];
                        const float4 g0 = row[0], g1 = row[1], g2 = row[2];
                        // a = sum_ii wx g, b = sum_ii ii wx g along the row
                        float2 axy = __fmul2_rn(w0, make_float2(g0.x, g0.y));
                        axy = __ffma2_rn(w1, make_float2(g1.x, g1.y), axy);
                        axy = __ffma2_rn(w2, make_float2(g2.x, g2.y), axy);
                        const float az = fmaf(wx[2], g2.z, fmaf(wx[1], g1.z, wx[0] * g0.z));
                        const float2 bxy = __ffma2_rn(w2d, make_float2(g2.x, g2.y), __fmul2_rn(w1, make_float2(g1.x, g1.y)));
                        const float bz = fmaf(w2d.x, g2.z, wx[1] * g1.z);
                        vxy = __ffma2_rn(wjk2, axy, vxy);
                        vzz = fmaf(wjk, az, vzz);
                        mxy = __ffma2_rn(wjk2, bxy, mxy);
                        mxz = fmaf(wjk, bz, mxz);
                        if (jj > 0) {
                            const float2 s2 = jj == 1 ? wjk2 : __fadd2_rn(wjk2, wjk2);
                            myy = __ffma2_rn(s2, axy, myy);
                            myz = fmaf(s2.x, az, myz);
                        }
                        if (kk > 0) {
                            const float2 s2 = kk == 1 ? wjk2 : __fadd2_rn(wjk2, wjk2);
                            mzy = __ffma2_rn(s2, axy, mzy);
                            mzz = fmaf(s2.x, az, mzz);
                        }
                    }
                }
                vx = vxy.x; vy = vxy.y; vz = vzz;
                // C = (4 / dx^2) sum w v (x_i - x_p)^T = (4 / dx) (moments - v f^T)   (Eq. 9)
                const float cs = 4.0f * P.inv_dx;
                const float2 cxy = __ffma2_rn(make_float2(-fx, -fx), vxy, mxy);
                const float2 cyy = __ffma2_rn(make_float2(-fy, -fy), vxy, myy);
                const float2 czy = __ffma2_rn(make_float2(-fz, -fz), vxy, mzy);
                Cm[0] = cs * cxy.x; Cm[1] = cs * cyy.x; Cm[2] = cs * czy.x;
                Cm[3] = cs * cxy.y; Cm[4] = cs * cyy.y; Cm[5] = cs * czy.y;
                Cm[6] = cs * fmaf(-fx, vzz, mxz); Cm[7] = cs * fmaf(-fy, vzz, myz); Cm[8] = cs * fmaf(-fz, vzz, mzz);
                // --- Eq. 4 and Eq. 10
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        Fn[3 * r + c] = F[3 * r + c] + P.dt * (Cm[3 * r] * F[c] + Cm[3 * r + 1] * F[3 + c] + Cm[3 * r + 2] * F[6 + c]);
                nxp = xi.x + P.dt * vx;
                nyp = xi.y + P.dt * vy;
                nzp = xi.z + P.dt * vz;
                // every value read from the slot has been consumed: refill it with the
                // next pass's particle
                if (pass + PD < npass && jn < total) prefetch_particle(s, in, ncand, jn, tid, ps);
                if (!finite3(nxp, nyp, nzp)) {
                    err |= kErrNumeric;
                    nxp = xi.x; nyp = xi.y; nzp = xi.z;
                }
                // --- stress of the new state (Eqs. 5-6) and the P2G inputs (Eqs. 1-3)
                float t[6];
                kirchhoff(Fn, ep.mu, ep.lam, t, err);
                const float kst = ep.stress_k, dxs = P.dx;
                float A[9] = {(m * Cm[0] - kst * t[0]) * dxs, (m * Cm[1] - kst * t[1]) * dxs, (m * Cm[2] - kst * t[2]) * dxs,
                              (m * Cm[3] - kst * t[1]) * dxs, (m * Cm[4] - kst * t[3]) * dxs, (m * Cm[5] - kst * t[4]) * dxs,
                              (m * Cm[6] - kst * t[2]) * dxs, (m * Cm[7] - kst * t[4]) * dxs, (m * Cm[8] - kst * t[5]) * dxs};
                int hx, hy, hz;
                const float ex = stencil_axis(nxp, P.inv_dx, n, hx, err);
                const float ey = stencil_axis(nyp, P.inv_dx, n, hy, err);
                const float ez = stencil_axis(nzp, P.inv_dx, n, hz, err);
                // q = m v - A' fx: the value at stencil offset o is q + A' o
                const float qx = m * vx - (A[0] * ex + A[1] * ey + A[2] * ez);
                const float qy = m * vy - (A[3] * ex + A[4] * ey + A[5] * ez);
                const float qz = m * vz - (A[6] * ex + A[7] * ey + A[8] * ez);
                if (!(isfinite(qx) && isfinite(qy) && isfinite(qz))) err |= kErrNumeric;
                const int ax0 = hx - ox, ay0 = hy - oy, az0 = hz - oz;
                const bool in_arena = ax0 >= 0 && ax0 <= 5 && ay0 >= 0 && ay0 <= 5 && az0 >= 0 && az0 <= 5;
                if (in_arena) {
                    // a base cell outside b (the particle moved into a neighbour
                    // block) widens the group's stencils beyond the 6^3 nodes of b
                    if (ax0 == 0 || ax0 == 5 || ay0 == 0 || ay0 == 5 || az0 == 0 || az0 == 5) s.wide = 1u;
                    const int abase = ax0 + kAy * ay0 + kAz * az0;
                    s.st_base[slot] = abase;
                    const uint32_t cls = (uint32_t)abase & 31u;
                    s.st_key[slot] = (uint16_t)(cls | (atomicAdd(&s.ccount[cls], 1u) << 5));
                    s.st_f[0][slot] = ex; s.st_f[1][slot] = ey; s.st_f[2][slot] = ez;
                    s.st_q[0][slot] = qx; s.st_q[1][slot] = qy; s.st_q[2][slot] = qz;
#pragma unroll
                    for (int q = 0; q < 9; ++q) s.st_a[q][slot] = A[q];
                    // bound of |q + A' o| over the stencil, per component
                    const float b0 = fabsf(qx) + 2.f * (fabsf(A[0]) + fabsf(A[1]) + fabsf(A[2]));
                    const float b1 = fabsf(qy) + 2.f * (fabsf(A[3]) + fabsf(A[4]) + fabsf(A[5]));
                    const float b2 = fabsf(qz) + 2.f * (fabsf(A[6]) + fabsf(A[7]) + fabsf(A[8]));
                    const float bp = fmaxf(fmaxf(b0, b1), b2);
                    atomicMax(&s.bmax, isfinite(bp) ? __float_as_uint(bp) : 0u);
                } else {
                    // moved further than one cell: scatter straight into G_{k+1}
                    s.st_base[slot] = -1;
                    float wx2[3], wy2[3], wz2[3];
                    bspline_weights(ex, wx2);
                    bspline_weights(ey, wy2);
                    bspline_weights(ez, wz2);
                    for (int kk = 0; kk < 3; ++kk)
                        for (int jj = 0; jj < 3; ++jj) {
                            const float wjk = wy2[jj] * wz2[kk];
                            const float rx = qx + A[1] * jj + A[2] * kk;
                            const float ry = qy + A[4] * jj + A[5] * kk;
                            const float rz = qz + A[7] * jj + A[8] * kk;
                            for (int ii = 0; ii < 3; ++ii) {
                                const float w = wx2[ii] * wjk;
                                red_add4(&Gnext[node_addr_env(env, hx + ii, hy + jj, hz + kk, nb, nbe)],
                                         make_float4(w * m, w * (rx + A[0] * ii), w * (ry + A[3] * ii), w * (rz + A[6] * ii)));
                            }
                        }
                    for (int c = 0; c < 8; ++c) {
                        const int gi = (hx + 2 * (c & 1)) >> 2, gj = (hy + (c & 2)) >> 2, gk = (hz + ((c >> 1) & 2)) >> 2;
                        mark_clear(B, eb0 + block_id(gi, gj, gk, nb), step + 1, m3n);
                    }
                }
                // --- destination block of the new state
                int ddx = (hx >> 2) - bx, ddy = (hy >> 2) - by, ddz = (hz >> 2) - bz;
                if (ddx < -1 || ddx > 1 || ddy < -1 || ddy > 1 || ddz < -1 || ddz > 1) {
                    err |= kErrCfl;
                    ddx = min(max(ddx, -1), 1); ddy = min(max(ddy, -1), 1); ddz = min(max(ddz, -1), 1);
                }
                d = (ddx + 1) + 3 * (ddy + 1) + 9 * (ddz + 1);
            } else {
                s.st_base[slot] = -1;
            }
            cp_async_commit();
            // --- stable rank by direction within the pass: per-warp counts, then
            // every warp derives the offsets it needs from the whole table (one
            // barrier per pass; warp 0 also publishes the pass's runs)
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
            uint8_t(*wc)[Smem::NWP] = s.wcnt[pass & 1];
            if (valid && rank == 0) wc[d][warp] = (uint8_t)__popc(peers);
            __syncthreads();
            const uint32_t out_base = s.out_base, chunk_first = s.chunk_first;
            uint32_t run = 0, before = 0;                 // lane l: pass total and earlier warps' count of direction l
            if (lane < 27) {
                // byte sums by one multiply (four counts of at most 32: no carries)
                auto bsum = [](uint32_t x) { return (x * 0x01010101u) >> 24; };
                if (Smem::NWP == 8) {
                    const uint2 c = *reinterpret_cast<const uint2 *>(&wc[lane][0]);
                    const uint32_t mlo = warp >= 4 ? 0xffffffffu : (1u << (8 * warp)) - 1u;
                    const uint32_t mhi = warp <= 4 ? 0u : (1u << (8 * (warp - 4))) - 1u;
                    run = bsum(c.x) + bsum(c.y);
                    before = bsum(c.x & mlo) + bsum(c.y & mhi);
                } else {
                    const uint32_t c = *reinterpret_cast<const uint32_t *>(&wc[lane][0]);
                    run = bsum(c);
                    before = bsum(c & ((1u << (8 * warp)) - 1u));
                }
            }
            uint32_t incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t my_off = __shfl_sync(0xffffffffu, incl - run + before, d & 31);
            // this warp's column of the other parity is next written by this warp, in
            // the next pass; every warp's reads of it ended before the barrier above
            if (lane < 28) s.wcnt[(pass + 1) & 1][lane][warp] = 0u;
            if (warp == 0 && chunk_first + pass < nchunk_cap) {
                const uint32_t pbase = out_base + pass * T;
                if (lane < 27) {
                    cout[chunk_first + pass].run[lane] = make_uint2(pbase + incl - run, run);
                    const int tx = bx + dir_dx(lane), ty = by + dir_dy(lane), tz = bz + dir_dz(lane);
                    if (run > 0u && tx >= 0 && ty >= 0 && tz >= 0 && tx < nb && ty < nb && tz < nb) {
                        uint4 *dst = inbox_out + (size_t)(eb0 + block_id(tx, ty, tz, nb)) * kInbox;
                        if (pass < (uint32_t)kNpMax)
                            dst[lane * kNpMax + pass] = make_uint4(pbase + incl - run, run, step + 1, 0u);
                        else
                            dst[kInbox - 1] = make_uint4(step + 1, 0u, 0u, 0u);   // overflow: use the run tables
                    }
                }
                const unsigned nz = __ballot_sync(0xffffffffu, lane < 27 && run > 0);
                if (lane == 0) s.mask |= nz;
            }
            const uint32_t pos = out_base + pass * T + my_off + rank;
            if (RECORD && valid && pos < nparticles) {
                rec.xi[pos] = xi;
                rec.f0[pos] = a0;
                rec.f1[pos] = a1;
                rec.f2[pos] = f2;
                store_vc(rec.vc, pos, vx, vy, vz, Cm);
                rec.src[pos] = source_slot(s, ncand, j);
            }
            if (valid && pos < nparticles) {
                out.xi[pos] = make_float4(nxp, nyp, nzp, idf);
                out.f0[pos] = make_float4(Fn[0], Fn[1], Fn[2], Fn[3]);
                out.f1[pos] = make_float4(Fn[4], Fn[5], Fn[6], Fn[7]);
                out.f2[pos] = Fn[8];
                if (WRITE_VC) store_vc(B.vc, pos, vx, vy, vz, Cm);
            }

            // --- P2G of the staged group (after every GP-th pass and the last one).
            // Lane l of warp w scatters staged slot 2 l + (w & 1) + 64 (w >> 1):
            // neighbouring lanes then hold particles of different cells.
            if (pass % GP == GP - 1 || pass + 1 == npass) {
                const int nstaged = (int)min((uint32_t)GROUP, total - (pass - pass % GP) * T);
                const float bmax = __uint_as_float(s.bmax);
                const bool wide = s.wide != 0u;
                const float sv = bmax > 0.f ? kFix / bmax : 1.0f;   // momentum fixed-point scale
                // order the group's arena particles by bank bucket (a counting sort over
                // 32 buckets): lane l of a warp then takes sorted position l * rows + j,
                // so the lanes of a warp sit in distinct banks at every stencil node
                const uint32_t cnt = s.ccount[lane];
                uint32_t cincl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, cincl, o);
                    if (lane >= o) cincl += y;
                }
                const uint32_t nin = __shfl_sync(0xffffffffu, cincl, 31);
                const uint32_t cexcl = cincl - cnt;
#pragma unroll
                for (int p = 0; p < GP; ++p) {
                    const int sl = p * T + tid;
                    const bool mine = sl < nstaged && s.st_base[sl] >= 0;
                    const uint32_t key = mine ? s.st_key[sl] : 0u;
                    const uint32_t off = __shfl_sync(0xffffffffu, cexcl, key & 31u);
                    if (mine) s.order[off + (key >> 5)] = (uint16_t)sl;
                }
                __syncthreads();
                const uint32_t rows = (nin + 31u) >> 5;
                for (uint32_t jr = warp; jr < rows; jr += NW) {
                    const uint32_t pos = lane * rows + jr;
                    if (pos >= nin) continue;
                    const int q = s.order[pos];
                    const int base = s.st_base[q];
                    if (base < 0) continue;
                    float wx[3], wy[3], wz[3];
                    bspline_weights(s.st_f[0][q], wx);
                    bspline_weights(s.st_f[1][q], wy);
                    bspline_weights(s.st_f[2][q], wz);
                    // momentum inputs in fixed-point units, as (x, y) and (z, mass)
                    // pairs for the packed f32x2 pipe: the value at stencil offset
                    // (ii, jj, kk) is q + A' (ii, jj, kk), the mass term the constant
                    // kFix (m_p 2^22 in mass units)
                    const float2 sv2 = make_float2(sv, sv), two = make_float2(2.f, 2.f);
                    const float2 qxy = __fmul2_rn(make_float2(s.st_q[0][q], s.st_q[1][q]), sv2);
                    const float2 qzm = make_float2(s.st_q[2][q] * sv, kFix);
                    const float2 aixy = __fmul2_rn(make_float2(s.st_a[0][q], s.st_a[3][q]), sv2);
                    const float2 ajxy = __fmul2_rn(make_float2(s.st_a[1][q], s.st_a[4][q]), sv2);
                    const float2 akxy = __fmul2_rn(make_float2(s.st_a[2][q], s.st_a[5][q]), sv2);
                    const float2 aizm = make_float2(s.st_a[6][q] * sv, 0.f);
                    const float2 ajzm = make_float2(s.st_a[7][q] * sv, 0.f);
                    const float2 akzm = make_float2(s.st_a[8][q] * sv, 0.f);
                    const float2 mm = make_float2(kMagic, kMagic);
                    const float2 wxx[3] = {make_float2(wx[0], wx[0]), make_float2(wx[1], wx[1]), make_float2(wx[2], wx[2])};
#pragma unroll
                    for (int kk = 0; kk < 3; ++kk) {
#pragma unroll
                        for (int jj = 0; jj < 3; ++jj) {
                            const float wjk = wy[jj] * wz[kk];
                            const float2 wjk2 = make_float2(wjk, wjk);
                            float2 rxy = qxy, rzm = qzm;
                            if (jj == 1) { rxy = __fadd2_rn(rxy, ajxy); rzm = __fadd2_rn(rzm, ajzm); }
                            if (jj == 2) { rxy = __ffma2_rn(two, ajxy, rxy); rzm = __ffma2_rn(two, ajzm, rzm); }
                            if (kk == 1) { rxy = __fadd2_rn(rxy, akxy); rzm = __fadd2_rn(rzm, akzm); }
                            if (kk == 2) { rxy = __ffma2_rn(two, akxy, rxy); rzm = __ffma2_rn(two, akzm, rzm); }
#pragma unroll
                            for (int ii = 0; ii < 3; ++ii) {
                                float2 vxy = rxy, vzm = rzm;
                                if (ii == 1) { vxy = __fadd2_rn(vxy, aixy); vzm = __fadd2_rn(vzm, aizm); }
                                if (ii == 2) { vxy = __ffma2_rn(two, aixy, vxy); vzm = __ffma2_rn(two, aizm, vzm); }
                                const float2 w2 = __fmul2_rn(wxx[ii], wjk2);
                                const float2 bxy = __ffma2_rn(w2, vxy, mm), bzm = __ffma2_rn(w2, vzm, mm);
                                const int a = base + ii + kAy * jj + kAz * kk;
                                atomicAdd(&s.acc[0][a], fix_round(bzm.y));
                                atomicAdd(&s.acc[1][a], fix_round(bxy.x));
                                atomicAdd(&s.acc[2][a], fix_round(bxy.y));
                                atomicAdd(&s.acc[3][a], fix_round(bzm.x));
                            }
                        }
                    }
                }
                __syncthreads();
                // arena -> G_{k+1}, then reset it for the next group: all 8^3 nodes,
                // or only the 6^3 around b when every base cell lies in b
                const float um = m / kFix, up = 1.0f / sv;
                const int nflush = wide ? 512 : 216;
                for (int q = tid; q < nflush; q += T) {
                    int lx8, ly8, lz8;
                    if (wide) {
                        lx8 = q & 7; ly8 = (q >> 3) & 7; lz8 = q >> 6;
                    } else {
                        lx8 = 1 + q % 6; ly8 = 1 + (q / 6) % 6; lz8 = 1 + q / 36;
                    }
                    const int a = lx8 + kAy * ly8 + kAz * lz8;
                    const int am = s.acc[0][a], px = s.acc[1][a], py = s.acc[2][a], pz = s.acc[3][a];
                    if (am != 0 || px != 0 || py != 0 || pz != 0) {
                        const int i = ox + lx8, jn = oy + ly8, k = oz + lz8;
                        if (i >= 0 && jn >= 0 && k >= 0 && i < n && jn < n && k < n)
                            red_add4(&Gnext[node_addr_env(env, i, jn, k, nb, nbe)],
                                     make_float4((float)am * um, (float)px * up, (float)py * up, (float)pz * up));
                        s.acc[0][a] = 0; s.acc[1][a] = 0; s.acc[2][a] = 0; s.acc[3][a] = 0;
                    }
                }
                // every thread read s.bmax, s.wide and the bucket sizes before the barriers
                // above; the next group's atomics come after the barrier below
                if (tid == 0) { s.bmax = 0; s.wide = 0; }
                if (tid < 32) s.ccount[tid] = 0u;
                __syncthreads();
            }
        }
        // the block's direction mask and size, read before warp 0 reuses them for the
        // next block
        const uint32_t mask_b = s.mask, total_b = s.total;
        cp_async_wait_all();
        __syncthreads();
        // blocks of the next sub-step (the last warp) and grid blocks to clear before
        // G_{k+1}'s reuse (the one before it): two chains of dependent global atomics
        // that run beside warp 0's set-up of the next block
        if (warp >= NW - 2 && lane < 27) {
            const int tx = bx + dir_dx(lane), ty = by + dir_dy(lane), tz = bz + dir_dz(lane);
            if (tx >= 0 && ty >= 0 && tz >= 0 && tx < nb && ty < nb && tz < nb) {
                const uint32_t tb = eb0 + block_id(tx, ty, tz, nb);
                if (warp == NW - 1 && ((mask_b >> lane) & 1u)) {
                    // heavy: b itself (lane 13) with more particles now than one pass
                    // of the CTA takes.  A neighbour's mark wins only for blocks that
                    // particles enter from outside, which are light.
                    if (atomicExch(&B.astamp[tb], step + 1) != step + 1) {
                        if (lane == 13 && total_b > (uint32_t)T)
                            act_next[atomicAdd(&ctrl->nactive[par ^ 1][0], 1u)] = tb;
                        else
                            act_next[acap - 1u - atomicAdd(&ctrl->nactive[par ^ 1][1], 1u)] = tb;
                    }
                }
                if (warp == NW - 2) mark_clear(B, tb, step + 1, m3n);
            }
        }
    }

    if (err) atomicOr(&ctrl->err, err);
    // last CTA: reset per-launch counters, advance the sub-step
    __syncthreads();
    // No fence before the done counter: the last CTA reads only part_alloc,
    // whose atomics every CTA consumed (its block's output range) before
    // counting itself done, and everything it writes is read by the next
    // launch, after this one has completed.
    if (tid == 0) {
        const uint32_t prev = atomicAdd(&ctrl->done, 1u);
        if (prev == gridDim.x - 1) {
            __threadfence();
            if (*(volatile uint32_t *)&ctrl->part_alloc != nparticles) atomicOr(&ctrl->err, kErrCapacity);
            ctrl->work = 0;
            ctrl->part_alloc = 0;
            ctrl->chunk_alloc = 0;
            ctrl->nactive[par][0] = 0;
            ctrl->nactive[par][1] = 0;
            ctrl->nclear[m3c] = 0;
            ctrl->done = 0;
            if (RECORD) *rec.nact = nact;
            ctrl->step = step + 1;
        }
    }
}

template <int T, int GP, int MINB = kMinBlocks<T, GP>, int PD = 1>
void launch_variant(const DevParams &P, const FusedBufs &B, const ToolFrame *tools, bool write_vc, int grid,
                    cudaStream_t st) {
    const StepRecord none{};
    if (write_vc)
        k_fused_step<true, T, GP, MINB, false, PD><<<grid, T, sizeof(FusedSmem<T, GP, PD>), st>>>(P, B, tools, none);
    else
        k_fused_step<false, T, GP, MINB, false, PD><<<grid, T, sizeof(FusedSmem<T, GP, PD>), st>>>(P, B, tools, none);
}

template <int T, int GP, int MINB = kMinBlocks<T, GP>, int PD = 1>
int variant_occupancy() {
    const int bytes = (int)sizeof(FusedSmem<T, GP, PD>);
    cudaFuncSetAttribute(k_fused_step<true, T, GP, MINB, false, PD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_fused_step<false, T, GP, MINB, false, PD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    int a = 0, b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_fused_step<true, T, GP, MINB, false, PD>, T, bytes);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_fused_step<false, T, GP, MINB, false, PD>, T, bytes);
    return a < b ? a : b;
}

}  // namespace

void launch_fused_step(const DevParams &P, const FusedBufs &B, const ToolFrame *tools, bool write_vc, int grid,
                       int config, cudaStream_t st) {
    switch (config) {
    case 1: launch_variant<256, 1>(P, B, tools, write_vc, grid, st); break;
    case 2: launch_variant<128, 2, kMinBlocks<128, 2>, 2>(P, B, tools, write_vc, grid, st); break;
    case 3: launch_variant<128, 1>(P, B, tools, write_vc, grid, st); break;
    case 4: launch_variant<256, 2, 2, 2>(P, B, tools, write_vc, grid, st); break;   // 2 CTAs per SM, 128 registers
    default: launch_variant<256, 2>(P, B, tools, write_vc, grid, st); break;
    }
}

int fused_step_threads(int config) { return config == 2 || config == 3 ? 128 : 256; }

// The recording sub-step of the differentiable rollout: the configuration of
// 256 threads, 2 passes per flush and 2 CTAs per SM (128 registers).
int fused_record_occupancy() {
    constexpr int bytes = (int)sizeof(FusedSmem<256, 2>);
    cudaFuncSetAttribute(k_fused_step<false, 256, 2, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_fused_step<false, 256, 2, 2, true>, 256, bytes);
    return a;
}

void launch_fused_step_record(const DevParams &P, const FusedBufs &B, const ToolFrame *tools, const StepRecord &rec,
                              int grid, cudaStream_t st) {
    k_fused_step<false, 256, 2, 2, true><<<grid, 256, sizeof(FusedSmem<256, 2>), st>>>(P, B, tools, rec);
}

// Also opts the kernel into its dynamic shared memory size on the current
// device; called when a handle is created.
int fused_step_occupancy(int config) {
    switch (config) {
    case 1: return variant_occupancy<256, 1>();
    case 2: return variant_occupancy<128, 2, kMinBlocks<128, 2>, 2>();
    case 3: return variant_occupancy<128, 1>();
    case 4: return variant_occupancy<256, 2, 2, 2>();
    default: return variant_occupancy<256, 2>();
    }
}

}  // namespace gbmpm
