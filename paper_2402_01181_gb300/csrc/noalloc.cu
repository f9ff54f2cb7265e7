// noalloc.cu -- the stable block sort for callers that cannot allocate device
// memory.  Some hosts own every byte of the GPU through their own pool or a
// fixed budget, and code running inside them must not call cudaMalloc or
// cudaFree (or anything that does, such as a framework's allocator).  This
// entry point runs the same kernels as the sort inside mpm_load_particles but
// keeps its scratch in a file-scope device array that lives as long as the
// library is loaded.
#include <cuda_runtime.h>

#include <string>

#include "../../include/mpm.h"
#include "common.cuh"
#include "launch.h"

using namespace gbmpm;

namespace {

// Largest grid this entry point accepts: n_grid <= 256, i.e. 64^3 blocks.
constexpr uint32_t kMaxBlocks = 64u * 64u * 64u;
// Layout (32-bit words): Ctrl (224 words: seven 128-byte lines),
// counts[kMaxBlocks], cursor[kMaxBlocks], offsets[kMaxBlocks + 1], padding.
// About 3 MB per device.
constexpr size_t kCtrlWords = sizeof(Ctrl) / 4;
static_assert(kCtrlWords == 224, "Ctrl is seven 128-byte lines");
constexpr size_t kScratchWords = kCtrlWords + 3 * (size_t)kMaxBlocks + 64;

static __device__ __align__(256) uint32_t g_sort_scratch[kScratchWords];

mpm_status fail(mpm_status st, const std::string &msg) {
    set_last_error(msg.c_str());   // reported by mpm_last_error()
    return st;
}

// Device address of the scratch array in the current context.  Host code only
// sees a host-side stand-in for g_sort_scratch, so the address must come from
// cudaGetSymbolAddress with the device current.  It is looked up on every
// call, not cached: a host that drives the GPU through its own (non-primary)
// context, or that resets the device and so gets a fresh copy of the
// library's device code, has the array at a different address.  The first
// lookup in a context also loads the library's device code there.
mpm_status scratch_address(uint32_t **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess || !p)
        return fail(MPM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    *out = static_cast<uint32_t *>(p);
    return MPM_OK;
}

// keys[j] = block of sorted entry j, from the block offsets of the sort: one
// warp per block, its lanes writing consecutive entries of the block's segment
__global__ void k_fill_sorted_keys(const uint32_t *__restrict__ offsets, uint32_t m, uint32_t *__restrict__ keys) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < m; b += warps) {
        const uint32_t first = offsets[b], last = offsets[b + 1];
        for (uint32_t j = first + lane; j < last; j += 32u) keys[j] = b;
    }
}

}  // namespace

extern "C" mpm_status mpm_block_sort_noalloc(const float *x, int64_t n, int32_t n_grid, uint32_t *ids,
                                             uint32_t *keys, void *cuda_stream) {
    if (n_grid < 8 || n_grid > 256 || (n_grid & (n_grid - 1)) != 0)
        return fail(MPM_ERR_ARG, "mpm_block_sort_noalloc: n_grid must be a power of two in [8, 256] "
                                 "(the static scratch holds at most 64^3 blocks)");
    if (n < 0 || n > ((int64_t)1 << 30)) return fail(MPM_ERR_ARG, "mpm_block_sort_noalloc: n outside [0, 2^30]");
    if (n > 0 && (!x || !ids || !keys)) return fail(MPM_ERR_ARG, "mpm_block_sort_noalloc: NULL pointer");
    if (n == 0) return MPM_OK;
    uint32_t *base = nullptr;
    mpm_status st = scratch_address(&base);
    if (st != MPM_OK) return st;
    const cudaStream_t stream = (cudaStream_t)cuda_stream;
    const uint32_t nb = (uint32_t)n_grid / 4u, m = nb * nb * nb;
    DevParams P{};
    P.n = n_grid;
    P.nb = (int)nb;
    P.nbe = m;
    P.n_envs = 1;
    P.dx = 1.0f / (float)n_grid;
    P.inv_dx = (float)n_grid;
    Ctrl *ctrl = reinterpret_cast<Ctrl *>(base);
    SortScratch s{};
    s.keys = keys;                              // caller's output
    s.perm = ids;                               // caller's output
    s.counts = base + kCtrlWords;
    s.cursor = s.counts + kMaxBlocks;
    s.offsets = s.cursor + kMaxBlocks;

    // the array keeps the previous call's contents: clear the counters and the error word
    cudaError_t e = cudaMemsetAsync(base, 0, (kCtrlWords + m) * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return fail(MPM_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    int sms = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    launch_block_sort(P, x, (uint32_t)n, s, ctrl, (sms > 0 ? sms : 1) * 8, stream);
    // the sort leaves keys as scratch; the output lists each sorted entry's key
    k_fill_sorted_keys<<<(sms > 0 ? sms : 1) * 8, 256, 0, stream>>>(s.offsets, m, keys);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MPM_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(MPM_ERR_CUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e));
    uint32_t err = 0;
    e = cudaMemcpy(&err, &ctrl->err, sizeof err, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(MPM_ERR_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
    if (err & kErrNumeric) return fail(MPM_ERR_NUMERIC, "mpm_block_sort_noalloc: non-finite position");
    if (err & kErrDomain) return fail(MPM_ERR_DOMAIN, "mpm_block_sort_noalloc: a stencil left the grid (clamped)");
    return MPM_OK;
}
