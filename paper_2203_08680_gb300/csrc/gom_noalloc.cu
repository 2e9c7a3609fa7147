// gom_noalloc.cu -- full fitness evaluation of a caller-given population with
// no device allocation at all: the scratch (the population packed into
// 32-individual words) is a fixed array in this file, resident on every GPU
// that loads the library.  For callers that cannot allocate device memory.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/gom.h"

namespace {

// Scratch: packed population, one 32-bit word per (variable, 32 individuals).
constexpr int64_t kNoAllocWords = GOM_NOALLOC_MAX_WORDS;
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
uint32_t *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device; the host-side symbol is not a device address).
cudaError_t scratch_address(uint32_t **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Packs pop[i*n + v] (uint8 {0,1}) into words[v*W + w], bit b = individual
// 32w + b; bits of individuals >= p are zero, so every word is rewritten.
__global__ void k_noalloc_pack(const uint8_t *pop, int32_t n, int32_t p, int32_t W, uint32_t *words)
{
    const int64_t total = static_cast<int64_t>(n) * W;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t v = idx / W;
        const int w = static_cast<int>(idx - v * W);
        uint32_t word = 0;
        for (int b = 0; b < 32; ++b) {
            const int64_t i = 32 * static_cast<int64_t>(w) + b;
            if (i < p && pop[i * n + v]) word |= 1u << b;
        }
        words[idx] = word;
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
    if (!d_row_ptr || !d_pop || !d_fitness_out || num_vertices < 1 || pop < 1) return GOM_E_ARG;
    if (pop > GOM_MAX_POPULATION) return GOM_E_LIMIT;
    int W = 1;
    while (32 * W < pop) W <<= 1;
    if (static_cast<int64_t>(num_vertices) * W > kNoAllocWords) return GOM_E_LIMIT;
    uint32_t *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return GOM_E_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (cudaMemsetAsync(d_fitness_out, 0, sizeof(int64_t) * pop, s) != cudaSuccess) return GOM_E_CUDA;
    const int64_t words = static_cast<int64_t>(num_vertices) * W;
    const int pack_grid = static_cast<int>((words + 255) / 256 < 4096 ? (words + 255) / 256 : 4096);
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
