// gom_noalloc.cu -- full fitness evaluation of a caller-given population with
// no device allocation at all: the scratch (the population packed into
// 32-individual words) is a fixed array in this file, resident on every GPU
// that loads the library.  For callers that cannot allocate device memory.
#include <cstdint>
#include <mutex>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/gom.h"

namespace {

// Scratch: packed population, one 32-bit word per (variable, 32 individuals).
constexpr int64_t kNoAllocWords = GOM_NOALLOC_MAX_WORDS;
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

// The scratch array's device address is valid only in the CUDA context it was
// looked up in, so the set-up is cached per context, keyed by the context's
// unique id (never reused within a process, unlike the CUcontext handle or
// the device number: a context made after cudaDeviceReset, or one the caller
// made current itself, gets a new id and a new look-up).
constexpr int kCacheSlots = 64;
struct ScratchSlot {
    unsigned long long ctx_id;
    uint32_t *ptr;
};
std::mutex g_setup_mutex;
ScratchSlot g_slots[kCacheSlots] = {};
int g_nslots = 0;
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

// Id of the current context.  With none current on this thread, the current
// device's primary context is made current first (cudaSetDevice does that and
// allocates nothing); a context the caller made current is left in place.
cudaError_t current_context_id(unsigned long long *id)
{
    cudaError_t e = cudaSuccess;
    if (!g_ctx_current || !g_ctx_id) {
        cudaDriverEntryPointQueryResult q1{}, q2{};
        void *f1 = nullptr, *f2 = nullptr;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess || q1 != cudaDriverEntryPointSuccess) return cudaErrorNotSupported;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess || q2 != cudaDriverEntryPointSuccess) return cudaErrorNotSupported;
        g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        g_ctx_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    if (!ctx) {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaSetDevice(dev);
        if (e != cudaSuccess) return e;
        if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
    }
    if (g_ctx_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

// Device address of the scratch array in the current context: looked up with
// cudaGetSymbolAddress the first time a context calls (the host-side symbol
// is not a device address), then taken from the cache.
cudaError_t scratch_address(uint32_t **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long id = 0;
    cudaError_t e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    for (int s = 0; s < g_nslots; ++s)
        if (g_slots[s].ctx_id == id) {
            *out = g_slots[s].ptr;
            return cudaSuccess;
        }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    // a full cache keeps working: the slot the id hashes to is replaced
    const int s = g_nslots < kCacheSlots ? g_nslots++ : static_cast<int>(id % kCacheSlots);
    g_slots[s] = ScratchSlot{id, static_cast<uint32_t *>(p)};
    *out = static_cast<uint32_t *>(p);
    return cudaSuccess;
}

// Packs pop[i*n + v] (uint8 {0,1}) into words[v*W + w], bit b = individual
// 32w + b; bits of individuals >= p are zero, so every word is rewritten.  A
// warp takes 32 variables of one word: lane l owns variable v0 + l, and for
// each of the 32 individuals the warp reads 32 consecutive bytes of its row.
__global__ void k_noalloc_pack(const uint8_t *pop, int32_t n, int32_t p, int32_t W, uint32_t *words)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const int64_t nchunks = (n + 31) / 32;
    for (int64_t it = warp; it < nchunks * W; it += nwarps) {
        const int64_t v = 32 * (it / W) + lane;
        const int w = static_cast<int>(it % W);
        uint32_t word = 0;
        if (v < n) {
            const int bmax = p - 32 * w < 32 ? p - 32 * w : 32;
            for (int b = 0; b < bmax; ++b)
                if (pop[(32 * static_cast<int64_t>(w) + b) * n + v]) word |= 1u << b;
            words[v * W + w] = word;
        }
    }
}

// fit[i] += sum over edges {u < v} of w_uv [x_u != x_v] (the cut weight):
// warps take 32-vertex chunks of one word, lane = individual.  The warp
// count of the grid is a multiple of W.
__global__ void k_noalloc_cut(const uint32_t *words, int32_t n, int32_t p, int32_t W, const int64_t *row_ptr,
                              const int32_t *col, const int32_t *wgt, int64_t *fit)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const int w = static_cast<int>(warp % W);
    const int64_t nchunks = (n + 31) / 32;
    long long acc = 0;
    for (int64_t ch = warp / W; ch < nchunks; ch += nwarps / W) {
        const int64_t uend = ch * 32 + 32 < n ? ch * 32 + 32 : n;
        for (int64_t u = 32 * ch; u < uend; ++u) {
            const uint32_t xu = words[u * W + w];
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                const int64_t v = col[e];
                if (v > u && (((xu ^ words[v * W + w]) >> lane) & 1u)) acc += wgt[e];
            }
        }
    }
    const int64_t i = 32 * static_cast<int64_t>(w) + lane;
    if (i < p && acc) atomicAdd(reinterpret_cast<unsigned long long *>(&fit[i]), static_cast<unsigned long long>(acc));
}

} // namespace

extern "C" int gom_fitness_noalloc(const int64_t *d_row_ptr, const int32_t *d_col, const int32_t *d_weight,
                                   int32_t num_vertices, const uint8_t *d_pop, int32_t pop,
                                   int64_t *d_fitness_out, void *cuda_stream)
{
    if (!d_row_ptr || !d_col || !d_weight || !d_pop || !d_fitness_out || num_vertices < 1 || pop < 1)
        return GOM_E_ARG;
    if (pop > GOM_MAX_POPULATION) return GOM_E_LIMIT;
    int W = 1;
    while (32 * W < pop) W <<= 1;
    if (static_cast<int64_t>(num_vertices) * W > kNoAllocWords) return GOM_E_LIMIT;
    uint32_t *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return GOM_E_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (cudaMemsetAsync(d_fitness_out, 0, sizeof(int64_t) * pop, s) != cudaSuccess) return GOM_E_CUDA;
    const int64_t pack_warps = (num_vertices + 31) / 32 * W;
    const int pack_grid = static_cast<int>((pack_warps + 7) / 8 < 4096 ? (pack_warps + 7) / 8 : 4096);
    k_noalloc_pack<<<pack_grid, 256, 0, s>>>(d_pop, num_vertices, pop, W, scratch);
    if (cudaGetLastError() != cudaSuccess) return GOM_E_CUDA;
    // 8 warps per block; the block count is a multiple of W / 8 so the warp count is a multiple of W
    const int mult = W > 8 ? W / 8 : 1;
    int cut_grid = static_cast<int>(((num_vertices + 31) / 32 * W + 7) / 8);
    cut_grid = cut_grid < 1024 ? cut_grid : 1024;
    cut_grid = (cut_grid + mult - 1) / mult * mult;
    k_noalloc_cut<<<cut_grid, 256, 0, s>>>(scratch, num_vertices, pop, W, d_row_ptr, d_col, d_weight,
                                           d_fitness_out);
    if (cudaGetLastError() != cudaSuccess) return GOM_E_CUDA;
    return GOM_OK;
}
