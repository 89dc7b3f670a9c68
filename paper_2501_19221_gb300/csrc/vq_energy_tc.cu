// vq_energy_tc.cu -- exact readout energies of a dense instance on the
// tensor cores.
//
// The readout energy E(x) = sum_i x_i (d_i + sum_{j != i} q_ij x_j), with
// q_ij = round(Q_ij 2^S) for Q as given and d_i = round((Q_ii + c_i) 2^S), is
// an integer form (the QUBO objective of Sec. 2 in fixed point). Each q_ij
// is written in balanced base-256 digits, q = sum_k 256^k t_k with t_k in
// [-128, 127], and digit plane k holds the t_k of every coupling as BF16,
// which represents every integer of magnitude <= 256 exactly. With x in
// {0, 1}, also exact in BF16, every product is exact, and every partial sum
// of a row of plane k against x_r is an integer of magnitude at most 128 n,
// below 2^24 for the sizes taken here, which FP32 accumulation holds exactly.
// The field kernel of vq_tc.cu (field only, unit scale) therefore returns
// G_k[r][i] = sum_j t_k,ij x_rj without rounding, and
//
//     E_r = sum_i x_ri (d_i + sum_k 256^k G_k[r][i])
//
// is formed in 64-bit integers. The sums are taken modulo 2^64 (unsigned
// arithmetic), which is exact because the finished energy lies in range.
// Plane k's per-tile sums are added into the same parts[g][r] (g: tiles of 64
// rows) as the CUDA-core kernel of vq_dense.cu produces.
#include <cuda_bf16.h>

#include <algorithm>

#include "vq_internal.cuh"

namespace vq {

namespace {

constexpr int64_t kMinN = 1024;                      // below this the CUDA-core kernel is as fast
constexpr int64_t kMaxN = 65536;                     // 128 n stays well below 2^24
constexpr size_t kMaxPlaneBytes = size_t(16) << 30;  // digit planes held per context
constexpr int kMaxPlanes = 8;                        // |q| < 2^62 needs at most 8 digits

// 127 (1 + 256 + ... + 256^(L-1)): every integer of magnitude up to this has
// an L-digit balanced base-256 form
unsigned long long digit_bound(int L) {
    unsigned long long u = 0;
    for (int k = 0; k < L; ++k) u = (u << 8) | 1ull;
    return 127ull * u;
}

// max |q_ij| over the off-diagonal entries (one block per row)
template <typename QT>
__global__ void __launch_bounds__(256) k_qfix_absmax(int64_t n, const QT* __restrict__ Q, int shift,
                                                     unsigned long long* out) {
    __shared__ unsigned long long sh[256];
    const int64_t i = blockIdx.x;
    unsigned long long m = 0;
    for (int64_t j = threadIdx.x; j < n; j += 256) {
        if (j == i) continue;
        const int64_t q = vqd::qfix<QT>(Q[i * n + j], shift);
        const unsigned long long a = q < 0 ? 0ull - (unsigned long long)q : (unsigned long long)q;
        m = a > m ? a : m;
    }
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = sh[threadIdx.x] > sh[threadIdx.x + s] ? sh[threadIdx.x] : sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(out, sh[0]);
}

// plane k, row i, column j: digit k of q_ij (zero on the diagonal and in the
// K padding [n, n_pad)); a remainder left after the last digit sets *err
template <typename QT>
__global__ void __launch_bounds__(256) k_digit_planes(int64_t n, int64_t n_pad, const QT* __restrict__ Q, int shift,
                                                      int planes, __nv_bfloat16* __restrict__ out, int* err) {
    const int64_t i = blockIdx.x;
    for (int64_t j = threadIdx.x; j < n_pad; j += 256) {
        int64_t q = (j < n && j != i) ? vqd::qfix<QT>(Q[i * n + j], shift) : 0;
        for (int k = 0; k < planes; ++k) {
            const int64_t t = ((q & 255) ^ 128) - 128;   // in [-128, 127], q - t divisible by 256
            out[((int64_t)k * n + i) * n_pad + j] = __float2bfloat16_rn((float)t);
            q = (q - t) / 256;
        }
        if (q != 0) atomicOr(err, 1);
    }
}

// operand x_rj = [S_rj > 0] (or X_rj != 0) as BF16 [R][n_pad], zero padding
template <bool FROM_BYTES>
__global__ void k_xop(int64_t R, int64_t n, int64_t n_pad, const float* __restrict__ S, const uint8_t* __restrict__ X,
                      __nv_bfloat16* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= R * n_pad) return;
    const int64_t r = t / n_pad, j = t - r * n_pad;
    bool on = false;
    if (j < n) on = FROM_BYTES ? X[r * n + j] != 0 : S[r * n + j] > 0.0f;
    out[t] = __float2bfloat16_rn(on ? 1.0f : 0.0f);
}

// parts[g][r] (=, plane 0; +=, later planes) of sum over the 64 rows i of
// tile g of x_ri 256^k G_k[r][i] (+ x_ri d_i on plane 0). Block: 64 rows x 4
// replicas; the replica loop is uniform over the block.
template <bool FROM_BYTES>
__global__ void __launch_bounds__(256) k_plane_combine(int64_t R, int64_t n, int plane, const float* __restrict__ G,
                                                       const float* __restrict__ S, const uint8_t* __restrict__ X,
                                                       const int64_t* __restrict__ dfix, int64_t* __restrict__ parts) {
    __shared__ unsigned long long sh[8];
    const int li = threadIdx.x & 63, rq = threadIdx.x >> 6;
    const int64_t i = (int64_t)blockIdx.x * 64 + li;
    const int64_t d = (plane == 0 && i < n) ? __ldg(dfix + i) : 0;
    for (int64_t rb = blockIdx.y; rb * 4 < R; rb += gridDim.y) {
        const int64_t r = rb * 4 + rq;
        unsigned long long v = 0;
        if (i < n && r < R) {
            const int64_t p = r * n + i;
            const bool xi = FROM_BYTES ? X[p] != 0 : S[p] > 0.0f;
            if (xi) v = ((unsigned long long)__float2ll_rn(G[p]) << (8 * plane)) + (unsigned long long)d;
        }
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
        __syncthreads();
        if (li == 0 && r < R) {
            const unsigned long long tot = sh[2 * rq] + sh[2 * rq + 1];
            int64_t* pp = parts + (int64_t)blockIdx.x * R + r;
            *pp = (int64_t)(plane == 0 ? tot : (unsigned long long)*pp + tot);
        }
        __syncthreads();
    }
}

template <typename QT>
int build_planes(veloxq_ctx* ctx, const QT* q) {
    const int64_t n = ctx->n, np = tc_pad(n);
    cudaStream_t st = ctx->stream;
    DevBuf tmp;
    VQ_TRY(tmp.ensure(16));
    unsigned long long* mx = tmp.as<unsigned long long>();
    int* err = reinterpret_cast<int*>(mx + 1);
    VQ_CUDA(cudaMemsetAsync(tmp.p, 0, 16, st));
    k_qfix_absmax<QT><<<(unsigned)n, 256, 0, st>>>(n, q, ctx->energy_shift, mx);
    VQ_LAUNCH_CHECK("energy digit bound");
    unsigned long long hm = 0;
    VQ_CUDA(cudaMemcpyAsync(&hm, mx, sizeof(hm), cudaMemcpyDeviceToHost, st));
    VQ_CUDA(cudaStreamSynchronize(st));
    int L = 1;
    while (L < kMaxPlanes && hm > digit_bound(L)) ++L;
    const size_t bytes = sizeof(__nv_bfloat16) * (size_t)L * (size_t)n * (size_t)np;
    if (hm > digit_bound(L) || bytes > kMaxPlaneBytes) {
        ctx->eplanes = -1;   // the CUDA-core kernel serves this context
        return VELOXQ_OK;
    }
    VQ_TRY(ctx->eplane.ensure(bytes));
    k_digit_planes<QT><<<(unsigned)n, 256, 0, st>>>(n, np, q, ctx->energy_shift, L, ctx->eplane.as<__nv_bfloat16>(), err);
    VQ_LAUNCH_CHECK("energy digit planes");
    int herr = 0;
    VQ_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    VQ_CUDA(cudaStreamSynchronize(st));
    if (herr) return fail(VELOXQ_ECUDA, "internal: the energy digit planes do not cover the couplings");
    ctx->eplanes = L;
    return VELOXQ_OK;
}

}  // namespace

int tc_energy_prepare(veloxq_ctx* ctx, int64_t R) {
    if (!ctx->dense || ctx->n < kMinN || ctx->n > kMaxN || ctx->eplanes < 0 || R < 1) return VELOXQ_OK;
    if (ctx->eplanes == 0) {
        switch (ctx->qx_type) {
            case VELOXQ_I8: VQ_TRY(build_planes(ctx, ctx->qx.as<int8_t>())); break;
            case VELOXQ_I32: VQ_TRY(build_planes(ctx, ctx->qx.as<int32_t>())); break;
            case VELOXQ_F32: VQ_TRY(build_planes(ctx, ctx->qx.as<float>())); break;
            case VELOXQ_F64: VQ_TRY(build_planes(ctx, ctx->qx.as<double>())); break;
        }
        if (ctx->eplanes < 0) return VELOXQ_OK;
    }
    const int64_t n = ctx->n, np = tc_pad(n);
    VQ_TRY(ctx->exop.ensure(sizeof(__nv_bfloat16) * (size_t)R * (size_t)np));
    VQ_TRY(ctx->efield.ensure(sizeof(float) * (size_t)R * (size_t)n));
    VQ_TRY(ctx->errw.ensure(sizeof(int) * 4));
    return VELOXQ_OK;
}

bool tc_energy_ready(const veloxq_ctx* ctx, int64_t R) {
    const int64_t np = tc_pad(ctx->n);
    return ctx->eplanes > 0 && R >= 1 && R <= (int64_t(1) << 20) &&
           ctx->exop.bytes >= sizeof(__nv_bfloat16) * (size_t)R * (size_t)np &&
           ctx->efield.bytes >= sizeof(float) * (size_t)R * (size_t)ctx->n;
}

// Enqueues the planes' products and sums on ctx->stream (no allocation, so it
// may be captured). A bounded wait that gives up sets ctx->errw.
int tc_energy(veloxq_ctx* ctx, int64_t R, const float* S, const uint8_t* X, int64_t* parts, int* nparts) {
    const int64_t n = ctx->n, np = tc_pad(n);
    cudaStream_t st = ctx->stream;
    *nparts = (int)div_up(n, 64);
    __nv_bfloat16* xop = ctx->exop.as<__nv_bfloat16>();
    const int64_t total = R * np;
    if (X) k_xop<true><<<(unsigned)div_up(total, 256), 256, 0, st>>>(R, n, np, nullptr, X, xop);
    else k_xop<false><<<(unsigned)div_up(total, 256), 256, 0, st>>>(R, n, np, S, nullptr, xop);
    VQ_LAUNCH_CHECK("energy operand");
    CUtensorMap mx;
    VQ_TRY(tc_operand_map(&mx, xop, VELOXQ_PREC_BF16, R, np, false));
    const dim3 cg((unsigned)div_up(n, 64), (unsigned)std::min<int64_t>(div_up(R, 4), 65535));
    for (int k = 0; k < ctx->eplanes; ++k) {
        CUtensorMap mp;
        VQ_TRY(tc_operand_map(&mp, ctx->eplane.as<__nv_bfloat16>() + (size_t)k * n * np, VELOXQ_PREC_BF16, n, np, true));
        VQ_TRY(tc_field(ctx, VELOXQ_PREC_BF16, (int32_t)R, mp, mx, nullptr, ctx->efield.as<float>(),
                        ctx->errw.as<int>()));
        if (X)
            k_plane_combine<true><<<cg, 256, 0, st>>>(R, n, k, ctx->efield.as<float>(), nullptr, X,
                                                      ctx->dfix.as<int64_t>(), parts);
        else
            k_plane_combine<false><<<cg, 256, 0, st>>>(R, n, k, ctx->efield.as<float>(), S, nullptr,
                                                       ctx->dfix.as<int64_t>(), parts);
        VQ_LAUNCH_CHECK("energy plane sums");
    }
    return VELOXQ_OK;
}

}  // namespace vq
