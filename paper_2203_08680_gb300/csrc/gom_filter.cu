// gom_filter.cu -- the learned trial filter: training and evaluation kernels
// for its MLP (16 inputs, 64 ReLU units, one logit; bf16 weights, fp32
// accumulation), the filter workspace and its C ABI.  The features, the
// skip decision, the audits and the training log are made inside the mixing
// kernels (gom_kernels.cu); every change that is kept is still decided by the
// exact integer partial evaluation of Alg. 2.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gom_ctx.h"
#include "gom_internal.h"
#include "gom_kernels.cuh"

namespace {

constexpr int kNW1 = kFilterHidden * kFilterIn;              // 1024
constexpr int kNTheta = kNW1 + kFilterHidden + kFilterHidden + 1; // W1, b1, W2, b2: 1153
constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Byte offsets inside the filter workspace.
struct FilterLayout {
    size_t st, hist, skipped, w1, w2, theta, adam_m, adam_v, grad, loss, log_x, log_y, logit;
    size_t dirty, quiet, dec, act, act_ptr, wcnt, total;
};

// The select phase's warps: at most 64 resident warps per SM in any launch.
int64_t select_warps_cap(const gom_ctx *ctx) { return 64 * static_cast<int64_t>(ctx->sms); }

FilterLayout filter_layout(const gom_ctx *ctx, int64_t cap)
{
    const int64_t m = ctx->m;
    FilterLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + std::max<size_t>(bytes, 1));
        return at;
    };
    L.st = take(sizeof(GomFilterState));
    L.hist = take(sizeof(uint32_t) * 6 * static_cast<size_t>(m));
    L.skipped = take(static_cast<size_t>(m));
    L.w1 = take(sizeof(uint16_t) * kNW1);
    L.w2 = take(sizeof(uint16_t) * kFilterHidden);
    L.theta = take(sizeof(float) * kNTheta);
    L.adam_m = take(sizeof(float) * kNTheta);
    L.adam_v = take(sizeof(float) * kNTheta);
    L.grad = take(sizeof(float) * kNTheta);
    L.loss = take(sizeof(double));
    L.log_x = take(sizeof(uint16_t) * kFilterIn * static_cast<size_t>(cap));
    L.log_y = take(static_cast<size_t>(cap));
    L.logit = take(sizeof(float) * static_cast<size_t>(cap));
    L.dirty = take(static_cast<size_t>(ctx->n));
    L.quiet = take(static_cast<size_t>(m));
    L.dec = take(static_cast<size_t>(m));
    L.act = take(sizeof(int32_t) * static_cast<size_t>(m));
    L.act_ptr = take(sizeof(int32_t) * static_cast<size_t>(ctx->k + 1));
    L.wcnt = take(sizeof(uint32_t) * static_cast<size_t>(select_warps_cap(ctx)));
    L.total = off;
    return L;
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_bits(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// Gradient of the weighted logistic loss over the log: threads (group, h),
// 4 groups of 64 per block, each group one sample at a time; unit h of the
// sample's forward pass (bf16-rounded weights, fp32 sums), the group's logit
// from a shared-memory sum, then h's gradient terms kept in registers and
// added into grad[] (fp32) once per block.  loss[0] += the summed loss.
__global__ void __launch_bounds__(256) k_filter_grad(const uint16_t *X, const uint8_t *y, int64_t N,
                                                     const float *theta, float pos_weight, float *grad, double *loss)
{
    __shared__ float s_part[4][2];
    __shared__ float s_red[256];
    const int h = threadIdx.x & 63, grp = threadIdx.x >> 6, lane = threadIdx.x & 31;
    const float *W1 = theta, *b1 = theta + kNW1, *W2 = b1 + kFilterHidden, *b2 = W2 + kFilterHidden;
    float w1[kFilterIn];
#pragma unroll
    for (int k = 0; k < kFilterIn; ++k) w1[k] = bf16_round(W1[h * kFilterIn + k]);
    const float w2 = bf16_round(W2[h]);
    float g1[kFilterIn], gb1 = 0.f, gw2 = 0.f, gb2 = 0.f;
    double lsum = 0.0;
#pragma unroll
    for (int k = 0; k < kFilterIn; ++k) g1[k] = 0.f;
    for (int64_t base = (int64_t)blockIdx.x * 4; base < N; base += (int64_t)gridDim.x * 4) {
        const int64_t n = base + grp;
        const bool valid = n < N;
        float x[kFilterIn];
#pragma unroll
        for (int k = 0; k < kFilterIn; ++k) x[k] = valid ? bf16_bits(X[n * kFilterIn + k]) : 0.f;
        float z = b1[h];
#pragma unroll
        for (int k = 0; k < kFilterIn; ++k) z = fmaf(w1[k], x[k], z);
        const float a = fmaxf(z, 0.f);
        float part = w2 * a;
        for (int off = 16; off; off >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, off);
        if (lane == 0) s_part[grp][h >> 5] = part;
        __syncthreads();
        const float out = b2[0] + s_part[grp][0] + s_part[grp][1];
        __syncthreads();
        if (!valid) continue;
        const float t = y[n] ? 1.f : 0.f, wt = y[n] ? pos_weight : 1.f;
        const float sig = 1.f / (1.f + expf(-out));
        const float d = wt * (sig - t);
        if (h == 0) {
            // log(1 + exp(-|out|)) + max(out, 0) - t out, weighted
            lsum += (double)(wt * (log1pf(expf(-fabsf(out))) + fmaxf(out, 0.f) - t * out));
            gb2 += d;
        }
        gw2 += d * a;
        const float dz = z > 0.f ? d * w2 : 0.f;
        gb1 += dz;
#pragma unroll
        for (int k = 0; k < kFilterIn; ++k) g1[k] = fmaf(dz, x[k], g1[k]);
    }
    // sum the 4 groups' terms of unit h, then one atomic per parameter and block
    auto block_add = [&](float v, float *dst) {
        s_red[threadIdx.x] = v;
        __syncthreads();
        if (grp == 0) {
            const float sum = s_red[h] + s_red[64 + h] + s_red[128 + h] + s_red[192 + h];
            atomicAdd(dst, sum);
        }
        __syncthreads();
    };
    for (int k = 0; k < kFilterIn; ++k) block_add(g1[k], grad + h * kFilterIn + k);
    block_add(gb1, grad + kNW1 + h);
    block_add(gw2, grad + kNW1 + kFilterHidden + h);
    if (h == 0) atomicAdd(grad + kNW1 + 2 * kFilterHidden, gb2);
    if (h == 0 && lsum != 0.0) atomicAdd(loss, lsum);
}

// One Adam step (Kingma & Ba, 2015) on the fp32 parameters with the mean
// gradient, then the bf16 copies of W1 and W2 the mixing kernels read.
__global__ void k_filter_step(float *theta, float *m, float *v, const float *grad, float inv_n, float lr, int step,
                              uint16_t *w1, uint16_t *w2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNTheta) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float g = grad[i] * inv_n;
    m[i] = b1 * m[i] + (1.f - b1) * g;
    v[i] = b2 * v[i] + (1.f - b2) * g * g;
    const float mh = m[i] / (1.f - powf(b1, (float)step)), vh = v[i] / (1.f - powf(b2, (float)step));
    theta[i] -= lr * mh / (sqrtf(vh) + eps);
    if (i < kNW1) w1[i] = __bfloat16_as_ushort(__float2bfloat16_rn(theta[i]));
    else if (i >= kNW1 + kFilterHidden && i < kNW1 + 2 * kFilterHidden)
        w2[i - kNW1 - kFilterHidden] = __bfloat16_as_ushort(__float2bfloat16_rn(theta[i]));
}

// The bf16 copies of W1 and W2 from the fp32 parameters (round to nearest even).
__global__ void k_filter_bf16(const float *theta, uint16_t *w1, uint16_t *w2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNW1) w1[i] = __bfloat16_as_ushort(__float2bfloat16_rn(theta[i]));
    else if (i >= kNW1 + kFilterHidden && i < kNW1 + 2 * kFilterHidden)
        w2[i - kNW1 - kFilterHidden] = __bfloat16_as_ushort(__float2bfloat16_rn(theta[i]));
}

// Logit of every logged sample, with the bf16 weights the select phase uses
// and its summation order (one thread per sample: unit h's sum over k from
// its bias, then the output's sum over h from zero, then the output bias).
__global__ void k_filter_eval(const uint16_t *X, int64_t N, const uint16_t *w1, const float *theta,
                              const uint16_t *w2, float *logit)
{
    const float *b1 = theta + kNW1, *b2 = theta + kNW1 + 2 * kFilterHidden;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        float x[kFilterIn];
#pragma unroll
        for (int k = 0; k < kFilterIn; ++k) x[k] = bf16_bits(X[n * kFilterIn + k]);
        float out = 0.f;
        for (int h = 0; h < kFilterHidden; ++h) {
            float z = b1[h];
#pragma unroll
            for (int k = 0; k < kFilterIn; ++k) z = fmaf(bf16_bits(w1[h * kFilterIn + k]), x[k], z);
            out = fmaf(bf16_bits(w2[h]), fmaxf(z, 0.f), out);
        }
        logit[n] = out + b2[0];
    }
}

// Deterministic initial weights: He-scaled uniform values from a SplitMix64
// stream (the initialisation is not part of the method).
void init_theta(std::vector<float> &theta, uint64_t seed)
{
    uint64_t x = seed;
    auto next = [&]() {
        uint64_t z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto unif = [&]() { return static_cast<float>((next() >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f; };
    theta.assign(kNTheta, 0.f);
    const float s1 = std::sqrt(6.f / kFilterIn), s2 = std::sqrt(6.f / kFilterHidden);
    for (int i = 0; i < kNW1; ++i) theta[i] = s1 * unif();
    for (int i = 0; i < kFilterHidden; ++i) theta[kNW1 + kFilterHidden + i] = s2 * unif();
}

} // namespace

extern "C" {

size_t gom_filter_workspace_bytes(gom_ctx_t *ctx, int64_t log_capacity)
{
    if (!ctx || log_capacity < 0) return 0;
    return filter_layout(ctx, log_capacity).total;
}

int gom_filter_attach(gom_ctx_t *ctx, void *d_workspace, size_t ws_bytes, int64_t log_capacity)
{
    if (!ctx || log_capacity < 0) return GOM_E_ARG;
    const FilterLayout L = filter_layout(ctx, log_capacity);
    if (!d_workspace || ws_bytes < L.total || reinterpret_cast<uintptr_t>(d_workspace) % kAlign)
        return GOM_E_WORKSPACE;
    char *base = static_cast<char *>(d_workspace);
    GOM_CUDA(ctx, cudaMemsetAsync(base, 0, L.total, ctx->stream));
    GomFilter &F = ctx->prm.flt;
    F.st = reinterpret_cast<GomFilterState *>(base + L.st);
    F.hist = reinterpret_cast<uint32_t *>(base + L.hist);
    F.skipped = reinterpret_cast<uint8_t *>(base + L.skipped);
    F.w1 = reinterpret_cast<const uint16_t *>(base + L.w1);
    F.b1 = reinterpret_cast<const float *>(base + L.theta) + kNW1;
    F.w2 = reinterpret_cast<const uint16_t *>(base + L.w2);
    F.b2 = reinterpret_cast<const float *>(base + L.theta) + kNW1 + 2 * kFilterHidden;
    F.log_x = reinterpret_cast<uint16_t *>(base + L.log_x);
    F.log_y = reinterpret_cast<uint8_t *>(base + L.log_y);
    F.log_cap = log_capacity;
    F.dirty = reinterpret_cast<uint8_t *>(base + L.dirty);
    F.quiet = reinterpret_cast<uint8_t *>(base + L.quiet);
    F.dec = reinterpret_cast<uint8_t *>(base + L.dec);
    F.act = reinterpret_cast<int32_t *>(base + L.act);
    F.act_ptr = reinterpret_cast<int32_t *>(base + L.act_ptr);
    F.wcnt = reinterpret_cast<uint32_t *>(base + L.wcnt);
    ctx->filter_base = base;
    ctx->filter_cap = log_capacity;
    GomFilterState st{};
    st.enabled = 0;
    st.disabled_at = -1;
    st.threshold = -INFINITY;
    st.min_recall = 0.5f;
    st.target_recall = 0.9f;
    st.low_streak = 0;
    GOM_CUDA(ctx, cudaMemcpyAsync(F.st, &st, sizeof(st), cudaMemcpyHostToDevice, ctx->stream));
    GOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->prm.learn = 0;
    return rebuild_graphs(ctx);
}

int gom_filter_set_mode(gom_ctx_t *ctx, int32_t mode)
{
    if (!ctx || mode < 0 || mode > 2) return GOM_E_ARG;
    if (mode > 0 && !ctx->filter_base) return GOM_E_STATE;
    // the change marks compare O with P, which the stage-all mode does not keep
    if (mode > 0 && ctx->prm.stage_all && ctx->persistent) return GOM_E_STATE;
    // the kernel instances with (or without) the filter's bookkeeping, on the same grids
    const bool learn = mode > 0;
    const void *mix = gom_mix_kernel(ctx->wpi, ctx->variant, learn);
    const void *run = gom_run_kernel(ctx->wpi, ctx->variant, learn);
    if (!mix || !run) return GOM_E_LIMIT; // no filter instances for elements of more than 64 variables
    GOM_CUDA(ctx, raise_smem_limit(mix, ctx->mix_smem));
    if (ctx->can_persist) {
        GOM_CUDA(ctx, raise_smem_limit(run, ctx->run_smem));
        int occ = 0;
        GOM_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, run, ctx->mix_threads, ctx->run_smem));
        if (static_cast<int64_t>(occ) * ctx->sms < ctx->grid_run) return GOM_E_STATE;
    }
    if (mode > 0) {
        const int32_t on = mode == 2 ? 1 : 0;
        GOM_CUDA(ctx, cudaMemcpyAsync(&ctx->prm.flt.st->enabled, &on, sizeof(on), cudaMemcpyHostToDevice,
                                      ctx->stream));
        GOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    ctx->mix_fn = mix;
    ctx->run_fn = run;
    if (ctx->bs_ok) { // the bit-sliced instances with (or without) the filter's select phase and bookkeeping
        ctx->run_bs_fn = gom_run_bs_kernel(ctx->bs_r, learn);
        ctx->mix_bs_fn = gom_mix_bs_kernel(ctx->bs_r, learn);
    }
    ctx->prm.learn = mode;
    return rebuild_graphs(ctx);
}

int gom_filter_configure(gom_ctx_t *ctx, float threshold, float target_recall, float min_recall)
{
    if (!ctx || !ctx->filter_base || !(min_recall >= 0.f && min_recall <= 1.f) ||
        !(target_recall >= 0.f && target_recall <= 1.f))
        return GOM_E_ARG;
    GomFilterState *st = ctx->prm.flt.st;
    const int32_t zero = 0;
    GOM_CUDA(ctx, cudaMemcpyAsync(&st->threshold, &threshold, sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    GOM_CUDA(ctx, cudaMemcpyAsync(&st->target_recall, &target_recall, sizeof(float), cudaMemcpyHostToDevice,
                                  ctx->stream));
    GOM_CUDA(ctx, cudaMemcpyAsync(&st->min_recall, &min_recall, sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    GOM_CUDA(ctx, cudaMemcpyAsync(&st->low_streak, &zero, sizeof(zero), cudaMemcpyHostToDevice, ctx->stream));
    GOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return GOM_OK;
}

int gom_filter_train(gom_ctx_t *ctx, int32_t epochs, float learning_rate, float pos_weight, float target_recall,
                     uint64_t seed, gom_filter_train_t *out)
{
    if (!ctx || !ctx->filter_base || epochs < 1 || !(learning_rate > 0.f) || !(pos_weight > 0.f) ||
        !(target_recall > 0.f && target_recall <= 1.f))
        return GOM_E_ARG;
    const FilterLayout L = filter_layout(ctx, ctx->filter_cap);
    char *base = ctx->filter_base;
    cudaStream_t s = ctx->stream;
    GomFilterState st{};
    GOM_CUDA(ctx, cudaMemcpyAsync(&st, ctx->prm.flt.st, sizeof(st), cudaMemcpyDeviceToHost, s));
    GOM_CUDA(ctx, cudaStreamSynchronize(s));
    const int64_t N = std::min<int64_t>(static_cast<int64_t>(st.log_count), ctx->filter_cap);
    if (N < 1) return GOM_E_STATE;
    std::vector<float> theta;
    init_theta(theta, seed);
    float *d_theta = reinterpret_cast<float *>(base + L.theta);
    float *d_m = reinterpret_cast<float *>(base + L.adam_m);
    float *d_v = reinterpret_cast<float *>(base + L.adam_v);
    float *d_grad = reinterpret_cast<float *>(base + L.grad);
    double *d_loss = reinterpret_cast<double *>(base + L.loss);
    uint16_t *d_w1 = reinterpret_cast<uint16_t *>(base + L.w1);
    uint16_t *d_w2 = reinterpret_cast<uint16_t *>(base + L.w2);
    const uint16_t *d_x = reinterpret_cast<const uint16_t *>(base + L.log_x);
    const uint8_t *d_y = reinterpret_cast<const uint8_t *>(base + L.log_y);
    float *d_logit = reinterpret_cast<float *>(base + L.logit);
    GOM_CUDA(ctx, cudaMemcpyAsync(d_theta, theta.data(), sizeof(float) * kNTheta, cudaMemcpyHostToDevice, s));
    GOM_CUDA(ctx, cudaMemsetAsync(d_m, 0, sizeof(float) * kNTheta, s));
    GOM_CUDA(ctx, cudaMemsetAsync(d_v, 0, sizeof(float) * kNTheta, s));
    const int grid = static_cast<int>(std::min<int64_t>((N + 3) / 4, static_cast<int64_t>(ctx->sms) * 8));
    double loss = 0.0;
    for (int e = 1; e <= epochs; ++e) {
        GOM_CUDA(ctx, cudaMemsetAsync(d_grad, 0, sizeof(float) * kNTheta, s));
        GOM_CUDA(ctx, cudaMemsetAsync(d_loss, 0, sizeof(double), s));
        k_filter_grad<<<grid, 256, 0, s>>>(d_x, d_y, N, d_theta, pos_weight, d_grad, d_loss);
        k_filter_step<<<(kNTheta + 255) / 256, 256, 0, s>>>(d_theta, d_m, d_v, d_grad, 1.f / static_cast<float>(N),
                                                            learning_rate, e, d_w1, d_w2);
        GOM_CUDA(ctx, cudaGetLastError());
        if (e == epochs) {
            GOM_CUDA(ctx, cudaMemcpyAsync(&loss, d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
        }
    }
    // the threshold: the largest logit that still keeps target_recall of the
    // useful logged samples above it (the bf16 weights, as the kernels use them)
    k_filter_eval<<<static_cast<int>(std::min<int64_t>((N + 7) / 8, 4096)), 256, 0, s>>>(d_x, N, d_w1, d_theta, d_w2,
                                                                                        d_logit);
    GOM_CUDA(ctx, cudaGetLastError());
    std::vector<float> logit(static_cast<size_t>(N));
    std::vector<uint8_t> label(static_cast<size_t>(N));
    GOM_CUDA(ctx, cudaMemcpyAsync(logit.data(), d_logit, sizeof(float) * N, cudaMemcpyDeviceToHost, s));
    GOM_CUDA(ctx, cudaMemcpyAsync(label.data(), d_y, static_cast<size_t>(N), cudaMemcpyDeviceToHost, s));
    GOM_CUDA(ctx, cudaStreamSynchronize(s));
    std::vector<float> pos;
    int64_t useful = 0;
    for (int64_t n = 0; n < N; ++n)
        if (label[n]) {
            pos.push_back(logit[n]);
            ++useful;
        }
    float thr = -INFINITY;
    if (!pos.empty()) {
        // skipping strictly below the (may_lose+1)-th smallest useful logit
        // loses at most may_lose useful samples, ties included
        std::sort(pos.begin(), pos.end());
        const int64_t may_lose = static_cast<int64_t>(std::floor((1.0 - target_recall) * useful));
        thr = pos[static_cast<size_t>(std::min<int64_t>(may_lose, useful - 1))];
    }
    int64_t skipped = 0, lost = 0;
    for (int64_t n = 0; n < N; ++n)
        if (logit[n] < thr) {
            ++skipped;
            lost += label[n];
        }
    GomFilterState *d_st = ctx->prm.flt.st;
    GOM_CUDA(ctx, cudaMemcpyAsync(&d_st->threshold, &thr, sizeof(float), cudaMemcpyHostToDevice, s));
    GOM_CUDA(ctx, cudaMemcpyAsync(&d_st->target_recall, &target_recall, sizeof(float), cudaMemcpyHostToDevice, s));
    GOM_CUDA(ctx, cudaStreamSynchronize(s));
    if (out) {
        out->samples = N;
        out->useful = useful;
        out->loss = loss / static_cast<double>(N);
        out->threshold = thr;
        out->skip_fraction = static_cast<double>(skipped) / static_cast<double>(N);
        out->recall = useful ? 1.0 - static_cast<double>(lost) / static_cast<double>(useful) : 1.0;
    }
    return GOM_OK;
}

int gom_filter_stats(gom_ctx_t *ctx, gom_filter_stats_t *out)
{
    if (!ctx || !out || !ctx->filter_base) return GOM_E_ARG;
    GomFilterState st{};
    GOM_CUDA(ctx, cudaMemcpyAsync(&st, ctx->prm.flt.st, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream));
    GOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::memset(out, 0, sizeof(*out));
    out->mode = ctx->prm.learn;
    out->enabled = st.enabled;
    out->disabled_at = st.disabled_at;
    out->threshold = st.threshold;
    out->log_count = static_cast<int64_t>(st.log_count);
    for (int x = 0; x < FC_N; ++x) {
        out->last[x] = static_cast<int64_t>(st.last[x]);
        out->total[x] = static_cast<int64_t>(st.total[x]);
    }
    return GOM_OK;
}

int gom_filter_get_params(gom_ctx_t *ctx, float *theta, float *adam_m, float *adam_v, float *grad)
{
    if (!ctx || !ctx->filter_base) return GOM_E_ARG;
    const FilterLayout L = filter_layout(ctx, ctx->filter_cap);
    char *base = ctx->filter_base;
    const size_t bytes = sizeof(float) * kNTheta;
    if (theta) GOM_CUDA(ctx, cudaMemcpyAsync(theta, base + L.theta, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    if (adam_m) GOM_CUDA(ctx, cudaMemcpyAsync(adam_m, base + L.adam_m, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    if (adam_v) GOM_CUDA(ctx, cudaMemcpyAsync(adam_v, base + L.adam_v, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    if (grad) GOM_CUDA(ctx, cudaMemcpyAsync(grad, base + L.grad, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    GOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return GOM_OK;
}

int gom_filter_set_params(gom_ctx_t *ctx, const float *theta, const float *adam_m, const float *adam_v)
{
    if (!ctx || !ctx->filter_base || !theta) return GOM_E_ARG;
    const FilterLayout L = filter_layout(ctx, ctx->filter_cap);
    char *base = ctx->filter_base;
    cudaStream_t s = ctx->stream;
    const size_t bytes = sizeof(float) * kNTheta;
    GOM_CUDA(ctx, cudaMemcpyAsync(base + L.theta, theta, bytes, cudaMemcpyHostToDevice, s));
    if (adam_m) GOM_CUDA(ctx, cudaMemcpyAsync(base + L.adam_m, adam_m, bytes, cudaMemcpyHostToDevice, s));
    else GOM_CUDA(ctx, cudaMemsetAsync(base + L.adam_m, 0, bytes, s));
    if (adam_v) GOM_CUDA(ctx, cudaMemcpyAsync(base + L.adam_v, adam_v, bytes, cudaMemcpyHostToDevice, s));
    else GOM_CUDA(ctx, cudaMemsetAsync(base + L.adam_v, 0, bytes, s));
    // the bf16 copies of W1 and W2, rounded as the training step writes them
    k_filter_bf16<<<(kNTheta + 255) / 256, 256, 0, s>>>(reinterpret_cast<const float *>(base + L.theta),
                                                        reinterpret_cast<uint16_t *>(base + L.w1),
                                                        reinterpret_cast<uint16_t *>(base + L.w2));
    GOM_CUDA(ctx, cudaGetLastError());
    GOM_CUDA(ctx, cudaStreamSynchronize(s));
    return GOM_OK;
}

int gom_filter_epoch(gom_ctx_t *ctx, float learning_rate, float pos_weight, int32_t step, double *loss)
{
    if (!ctx || !ctx->filter_base || !(learning_rate > 0.f) || !(pos_weight > 0.f) || step < 1) return GOM_E_ARG;
    const FilterLayout L = filter_layout(ctx, ctx->filter_cap);
    char *base = ctx->filter_base;
    cudaStream_t s = ctx->stream;
    GomFilterState st{};
    GOM_CUDA(ctx, cudaMemcpyAsync(&st, ctx->prm.flt.st, sizeof(st), cudaMemcpyDeviceToHost, s));
    GOM_CUDA(ctx, cudaStreamSynchronize(s));
    const int64_t N = std::min<int64_t>(static_cast<int64_t>(st.log_count), ctx->filter_cap);
    if (N < 1) return GOM_E_STATE;
    float *d_theta = reinterpret_cast<float *>(base + L.theta);
    float *d_grad = reinterpret_cast<float *>(base + L.grad);
    double *d_loss = reinterpret_cast<double *>(base + L.loss);
    const int grid = static_cast<int>(std::min<int64_t>((N + 3) / 4, static_cast<int64_t>(ctx->sms) * 8));
    GOM_CUDA(ctx, cudaMemsetAsync(d_grad, 0, sizeof(float) * kNTheta, s));
    GOM_CUDA(ctx, cudaMemsetAsync(d_loss, 0, sizeof(double), s));
    k_filter_grad<<<grid, 256, 0, s>>>(reinterpret_cast<const uint16_t *>(base + L.log_x),
                                       reinterpret_cast<const uint8_t *>(base + L.log_y), N, d_theta, pos_weight,
                                       d_grad, d_loss);
    k_filter_step<<<(kNTheta + 255) / 256, 256, 0, s>>>(d_theta, reinterpret_cast<float *>(base + L.adam_m),
                                                        reinterpret_cast<float *>(base + L.adam_v), d_grad,
                                                        1.f / static_cast<float>(N), learning_rate, step,
                                                        reinterpret_cast<uint16_t *>(base + L.w1),
                                                        reinterpret_cast<uint16_t *>(base + L.w2));
    GOM_CUDA(ctx, cudaGetLastError());
    double l = 0.0;
    GOM_CUDA(ctx, cudaMemcpyAsync(&l, d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    GOM_CUDA(ctx, cudaStreamSynchronize(s));
    if (loss) *loss = l / static_cast<double>(N);
    return GOM_OK;
}

int gom_filter_log(gom_ctx_t *ctx, int64_t max, uint16_t *x, uint8_t *y, int64_t *n)
{
    if (!ctx || !ctx->filter_base || max < 0 || !n) return GOM_E_ARG;
    const FilterLayout L = filter_layout(ctx, ctx->filter_cap);
    char *base = ctx->filter_base;
    GomFilterState st{};
    GOM_CUDA(ctx, cudaMemcpyAsync(&st, ctx->prm.flt.st, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream));
    GOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *n = std::min<int64_t>(static_cast<int64_t>(st.log_count), ctx->filter_cap);
    const int64_t c = std::min(*n, max);
    if (c > 0 && x)
        GOM_CUDA(ctx, cudaMemcpyAsync(x, base + L.log_x, sizeof(uint16_t) * kFilterIn * c, cudaMemcpyDeviceToHost,
                                      ctx->stream));
    if (c > 0 && y) GOM_CUDA(ctx, cudaMemcpyAsync(y, base + L.log_y, c, cudaMemcpyDeviceToHost, ctx->stream));
    GOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return GOM_OK;
}

int gom_filter_logits(gom_ctx_t *ctx, int64_t n, float *logits)
{
    if (!ctx || !ctx->filter_base || n < 0 || (n > 0 && !logits) || n > ctx->filter_cap) return GOM_E_ARG;
    if (n == 0) return GOM_OK;
    const FilterLayout L = filter_layout(ctx, ctx->filter_cap);
    char *base = ctx->filter_base;
    cudaStream_t s = ctx->stream;
    float *d_logit = reinterpret_cast<float *>(base + L.logit);
    k_filter_eval<<<static_cast<int>(std::min<int64_t>((n + 7) / 8, 4096)), 256, 0, s>>>(
        reinterpret_cast<const uint16_t *>(base + L.log_x), n, reinterpret_cast<const uint16_t *>(base + L.w1),
        reinterpret_cast<const float *>(base + L.theta), reinterpret_cast<const uint16_t *>(base + L.w2), d_logit);
    GOM_CUDA(ctx, cudaGetLastError());
    GOM_CUDA(ctx, cudaMemcpyAsync(logits, d_logit, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    GOM_CUDA(ctx, cudaStreamSynchronize(s));
    return GOM_OK;
}

int gom_filter_skipped(gom_ctx_t *ctx, uint8_t *host_mask)
{
    if (!ctx || !host_mask || !ctx->filter_base) return GOM_E_ARG;
    std::vector<uint8_t> byq(static_cast<size_t>(ctx->m));
    GOM_CUDA(ctx, cudaMemcpyAsync(byq.data(), ctx->prm.flt.skipped, static_cast<size_t>(ctx->m),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    GOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int64_t q = 0; q < ctx->m; ++q) host_mask[ctx->celems[q]] = byq[q];
    return GOM_OK;
}

} // extern "C"
