// vq_common.cu -- kernels shared by every path: Philox initial state, the
// per-replica best-so-far update, the bit readout of improved replicas, the
// argmin over replicas and the unpacking of the winner, energy totals.
#include <atomic>

#include "vq_internal.cuh"

namespace vq {

int device_sms(int device) {
    static std::atomic<int> cache[64];
    int v = (device >= 0 && device < 64) ? cache[device].load(std::memory_order_relaxed) : 0;
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v < 1) {
        cudaGetLastError();
        v = 1;
    }
    if (device >= 0 && device < 64) cache[device].store(v, std::memory_order_relaxed);
    return v;
}

namespace {

__global__ void k_init_state(int64_t n, int32_t R, uint64_t seed, float sigma0, int layout, float* S, float* Y) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = n * (int64_t)R;
    if (t >= total) return;
    int64_t i;
    int32_t r;
    if (layout == LAYOUT_RN) { r = (int32_t)(t / n); i = t - (int64_t)r * n; }
    else { i = t / R; r = (int32_t)(t - i * R); }
    float s, y;
    vqd::init_pair(i, r, seed, sigma0, &s, &y);
    S[t] = s;
    Y[t] = y;
}

// total_r = sum_g parts[g][r] (fixed order); keep the first strictly lower.
__global__ void k_best_update(int32_t R, int nparts, const int64_t* __restrict__ parts, int64_t* best,
                              uint8_t* improved) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    int64_t tot = 0;
    for (int g = 0; g < nparts; ++g) tot += parts[(int64_t)g * R + r];
    const bool better = tot < best[r];
    if (better) best[r] = tot;
    improved[r] = better ? 1 : 0;
}

// replica-major state: one warp per 32 consecutive variables of one replica
__global__ void k_best_bits_rn(int64_t n, int32_t R, const float* __restrict__ S, const uint8_t* __restrict__ improved,
                               uint32_t* bits) {
    const int64_t nw = (n + 31) / 32;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over R * nw * 32
    const int64_t r = t / (nw * 32);
    if (r >= R) return;
    const int64_t i = t - r * nw * 32;
    if (!improved[r]) return;            // uniform over the warp (nw*32 is a multiple of 32)
    const bool bit = i < n && S[r * n + i] > 0.0f;
    const uint32_t word = __ballot_sync(0xffffffffu, bit);
    if ((threadIdx.x & 31) == 0) bits[r * nw + (i >> 5)] = word;
}

// variable-major state: a thread makes one word (32 variables) of one
// replica; consecutive threads take consecutive replicas of the same word.
__global__ void k_best_bits_nr(int64_t n, int32_t R, const float* __restrict__ S, const uint8_t* __restrict__ improved,
                               uint32_t* bits) {
    const int64_t nw = (n + 31) / 32;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over nw * R
    const int64_t w = t / R;
    const int32_t r = (int32_t)(t - w * R);
    if (w >= nw || !improved[r]) return;
    uint32_t word = 0;
    for (int b = 0; b < 32; ++b) {
        const int64_t i = w * 32 + b;
        if (i < n && S[i * R + r] > 0.0f) word |= 1u << b;
    }
    bits[(int64_t)r * nw + w] = word;
}

// argmin over replicas (lowest index on ties) -> misc[0]
__global__ void k_argmin(int32_t R, const int64_t* __restrict__ best, int64_t* misc) {
    __shared__ int64_t sv[1024];
    __shared__ int32_t si[1024];
    int64_t bv = INT64_MAX;
    int32_t bi = INT32_MAX;
    for (int32_t r = threadIdx.x; r < R; r += blockDim.x) {
        const int64_t v = best[r];
        if (v < bv || (v == bv && r < bi)) { bv = v; bi = r; }
    }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const int64_t v = sv[threadIdx.x + s];
            const int32_t i = si[threadIdx.x + s];
            if (v < sv[threadIdx.x] || (v == sv[threadIdx.x] && i < si[threadIdx.x])) {
                sv[threadIdx.x] = v;
                si[threadIdx.x] = i;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        misc[0] = si[0];
        misc[1] = sv[0];
    }
}

__global__ void k_unpack(int64_t n, const uint32_t* __restrict__ bits, const int64_t* __restrict__ misc, uint8_t* x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t nw = (n + 31) / 32;
    const int64_t r = misc[0];
    x[i] = (uint8_t)((bits[r * nw + (i >> 5)] >> (i & 31)) & 1u);
}

// 32x32 tiles, numbered along one grid axis (either side may exceed the
// 65535 limit of the second axis: n ~ 1e8 variables by a few replicas).
__global__ void k_transpose(const float* __restrict__ in, float* __restrict__ out, int64_t rows, int64_t cols) {
    __shared__ float tile[32][33];
    const int64_t tcols = (cols + 31) / 32;
    const int64_t tr = (int64_t)blockIdx.x / tcols;
    const int64_t r0 = tr * 32, c0 = ((int64_t)blockIdx.x - tr * tcols) * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k, c = c0 + threadIdx.x;
        tile[k][threadIdx.x] = (r < rows && c < cols) ? in[r * cols + c] : 0.0f;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[c * rows + r] = tile[threadIdx.x][k];
    }
}

__global__ void k_sum_parts(int64_t B, int nparts, const int64_t* __restrict__ parts, int shift, double* E,
                            int64_t* E_int) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    int64_t tot = 0;
    for (int g = 0; g < nparts; ++g) tot += parts[(int64_t)g * B + b];
    if (E) E[b] = ldexp((double)tot, -shift);
    if (E_int) E_int[b] = tot >> shift;     // integer contexts: tot is a multiple of 2^shift
}

}  // namespace

int launch_init_state(veloxq_ctx* ctx, int32_t R, uint64_t seed, float sigma0, Layout layout, float* S, float* Y) {
    const int64_t total = ctx->n * (int64_t)R;
    if (total == 0) return VELOXQ_OK;
    k_init_state<<<(unsigned)div_up(total, 256), 256, 0, ctx->stream>>>(ctx->n, R, seed, sigma0, (int)layout, S, Y);
    VQ_LAUNCH_CHECK("init_state");
    return VELOXQ_OK;
}

int launch_transpose(cudaStream_t st, const float* in, float* out, int64_t rows, int64_t cols) {
    const int64_t tiles = div_up(cols, 32) * div_up(rows, 32);
    if (tiles == 0) return VELOXQ_OK;
    if (tiles > INT32_MAX) return fail(VELOXQ_EINVAL, "transpose: state too large");
    dim3 b(32, 8);
    k_transpose<<<(unsigned)tiles, b, 0, st>>>(in, out, rows, cols);
    VQ_LAUNCH_CHECK("transpose");
    return VELOXQ_OK;
}

int launch_best_update(veloxq_ctx* ctx, int32_t R, int nparts, const int64_t* parts, int64_t* best, uint8_t* improved) {
    k_best_update<<<(unsigned)div_up(R, 256), 256, 0, ctx->stream>>>(R, nparts, parts, best, improved);
    VQ_LAUNCH_CHECK("best_update");
    return VELOXQ_OK;
}

int launch_best_bits(veloxq_ctx* ctx, int32_t R, Layout layout, const float* S, const uint8_t* improved, uint32_t* bits) {
    const int64_t n = ctx->n, nw = (n + 31) / 32;
    if (layout == LAYOUT_RN) {
        const int64_t total = (int64_t)R * nw * 32;
        k_best_bits_rn<<<(unsigned)div_up(total, 256), 256, 0, ctx->stream>>>(n, R, S, improved, bits);
    } else {
        const int64_t total = (int64_t)R * nw;
        k_best_bits_nr<<<(unsigned)div_up(total, 256), 256, 0, ctx->stream>>>(n, R, S, improved, bits);
    }
    VQ_LAUNCH_CHECK("best_bits");
    return VELOXQ_OK;
}

int launch_argmin_unpack(veloxq_ctx* ctx, int32_t R, const int64_t* best, const uint32_t* bits, int64_t* misc,
                         uint8_t* x) {
    k_argmin<<<1, 1024, 0, ctx->stream>>>(R, best, misc);
    if (x) k_unpack<<<(unsigned)div_up(ctx->n, 256), 256, 0, ctx->stream>>>(ctx->n, bits, misc, x);
    VQ_LAUNCH_CHECK("argmin");
    return VELOXQ_OK;
}

int launch_sum_parts(veloxq_ctx* ctx, int64_t B, int nparts, const int64_t* parts, double* E, int64_t* E_int) {
    if (B == 0) return VELOXQ_OK;
    k_sum_parts<<<(unsigned)div_up(B, 128), 128, 0, ctx->stream>>>(B, nparts, parts, ctx->energy_shift, E, E_int);
    VQ_LAUNCH_CHECK("sum_parts");
    return VELOXQ_OK;
}

}  // namespace vq
