// vq_dense.cu -- dense instances on the CUDA cores (the plain FP32 form):
// F = S Qoff as a register-tiled SGEMM (M = replicas, N = K = n; S replica-major
// [R][n], Qoff symmetric row-major) with the ballistic-SB update fused into the
// epilogue, and the exact readout energy in int64 fixed point.
#include <algorithm>

#include "vq_internal.cuh"

namespace vq {

namespace {

constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;   // 256 threads, 8x8 outputs each
constexpr int BST = 4;   // stages of the Qoff tile when it is copied asynchronously

// 16-byte asynchronous copy global -> shared (cp.async, L2 only); the bytes
// past `bytes` (0 to 16) are zero-filled
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// C[r][i] = sum_j S[r][j] Qoff[j][i]. Tiles are zero-filled past the edges.
// With gridDim.z = ksplit > 1 (small problems: too few output tiles to fill
// the GPU) block z sums k-tiles [z per, (z+1) per) into part[z][r][i] and
// k_dense_finish adds the splits in order and applies the update.
// ASYNC (rows of Qoff 16-byte aligned, n % 4 == 0): the Qoff tiles come
// through BST stages of cp.async copies, three tiles ahead, so that their
// DRAM latency is hidden; the S tiles are staged through registers one tile
// ahead (they are transposed on the way). The sum of every output is taken
// in the same order either way.
template <bool FIELD_ONLY, bool ASYNC>
__global__ void __launch_bounds__(256) k_dense_step(int32_t R, int32_t n, const float* __restrict__ S_cur,
                                                    const float* __restrict__ Qoff, float* __restrict__ S_nxt,
                                                    float* __restrict__ Y, const float* __restrict__ bf,
                                                    const float* __restrict__ a_table, int k, float dt, float a0,
                                                    float c0, float* __restrict__ F_out, int method, float alpha,
                                                    int ktile_per, float* __restrict__ part) {
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[ASYNC ? BST : 2][BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
    // A tile: 128 rows x 8 k -> thread loads 4 consecutive k of one row
    const int a_row = tid / 2, a_k = (tid % 2) * 4;
    // B tile: 8 k x 128 cols -> thread loads 4 consecutive cols of one k
    const int b_k = tid / 32, b_col = (tid % 32) * 4;
    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.0f;

    auto load_tiles = [&](int kt, float (&ra)[4], float (&rb)[4]) {
        const int64_t gr = m0 + a_row;
        const int64_t gk = (int64_t)kt * BK + a_k;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            ra[q] = (gr < R && gk + q < n) ? vqd::field_operand(method, __ldg(S_cur + gr * n + gk + q)) : 0.0f;
        const int64_t bk = (int64_t)kt * BK + b_k;
        const int64_t bc = n0 + b_col;
#pragma unroll
        for (int q = 0; q < 4; ++q) rb[q] = (bk < n && bc + q < n) ? __ldg(Qoff + bk * n + bc + q) : 0.0f;
    };
    auto store_tiles = [&](int buf, const float (&ra)[4], const float (&rb)[4]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) As[buf][a_k + q][a_row] = ra[q];
        *reinterpret_cast<float4*>(&Bs[buf][b_k][b_col]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
    };

    const int ktiles = (int)div_up(n, BK);
    const int kt0 = (int)blockIdx.z * ktile_per, kt1 = min(ktiles, kt0 + ktile_per);
    float ra[4], rb[4];
    // the 8 k of one tile into acc
    auto compute = [&](const float (*A)[BM], const float (*Bt)[BN]) {
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float av[TM], bv[TN];
            const float4 a0v = *reinterpret_cast<const float4*>(&A[kk][ty * 4]);
            const float4 a1v = *reinterpret_cast<const float4*>(&A[kk][64 + ty * 4]);
            const float4 b0v = *reinterpret_cast<const float4*>(&Bt[kk][tx * 4]);
            const float4 b1v = *reinterpret_cast<const float4*>(&Bt[kk][64 + tx * 4]);
            av[0] = a0v.x; av[1] = a0v.y; av[2] = a0v.z; av[3] = a0v.w;
            av[4] = a1v.x; av[5] = a1v.y; av[6] = a1v.z; av[7] = a1v.w;
            bv[0] = b0v.x; bv[1] = b0v.y; bv[2] = b0v.z; bv[3] = b0v.w;
            bv[4] = b1v.x; bv[5] = b1v.y; bv[6] = b1v.z; bv[7] = b1v.w;
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
    };
    if constexpr (ASYNC) {
        auto load_a = [&](int kt, float (&r)[4]) {
            const int64_t gr = m0 + a_row;
            const int64_t gk = (int64_t)kt * BK + a_k;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                r[q] = (gr < R && gk + q < n) ? vqd::field_operand(method, __ldg(S_cur + gr * n + gk + q)) : 0.0f;
        };
        auto store_a = [&](int buf, const float (&r)[4]) {
#pragma unroll
            for (int q = 0; q < 4; ++q) As[buf][a_k + q][a_row] = r[q];
        };
        // this thread's 16 bytes of the Qoff tile kt: row kt BK + b_k, columns n0 + b_col ..
        auto issue_b = [&](int kt, int st) {
            const int64_t bk = (int64_t)kt * BK + b_k;
            const int64_t bc = n0 + b_col;
            const float* src = Qoff;
            int bytes = 0;
            if (bk < n && bc < n) {
                src = Qoff + bk * n + bc;
                bytes = (n - bc) >= 4 ? 16 : (int)((n - bc) * 4);
            }
            cp_async16(&Bs[st][b_k][b_col], src, bytes);
        };
        const int nk = kt1 - kt0;
#pragma unroll
        for (int st = 0; st < BST - 1; ++st) {
            if (st < nk) issue_b(kt0 + st, st);
            cp_async_commit();
        }
        if (nk > 0) {
            load_a(kt0, ra);
            store_a(0, ra);
        }
        for (int t = 0; t < nk; ++t) {
            cp_async_wait<BST - 2>();      // this thread's copies of tile t have landed
            __syncthreads();               // every copy of tile t and its S tile are visible; tile t - 1 is free
            if (t + BST - 1 < nk) issue_b(kt0 + t + BST - 1, (t + BST - 1) % BST);
            cp_async_commit();
            if (t + 1 < nk) load_a(kt0 + t + 1, ra);
            compute(As[t & 1], Bs[t % BST]);
            if (t + 1 < nk) store_a((t + 1) & 1, ra);
        }
        cp_async_wait<0>();
    } else {
    if (kt0 < kt1) {
        load_tiles(kt0, ra, rb);
        store_tiles(0, ra, rb);
    }
    __syncthreads();
    for (int kt = kt0; kt < kt1; ++kt) {
        const int cur = (kt - kt0) & 1;
        if (kt + 1 < kt1) load_tiles(kt + 1, ra, rb);
        compute(As[cur], Bs[cur]);
        if (kt + 1 < kt1) store_tiles(cur ^ 1, ra, rb);
        __syncthreads();
    }
    }
    if (gridDim.z > 1) {   // partial sums of this k-range; the update runs in k_dense_finish
        float* P = part + (int64_t)blockIdx.z * R * n;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int64_t r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
            if (r >= R) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int64_t c = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
                if (c < n) P[r * n + c] = acc[i][j];
            }
        }
        return;
    }
    // ---- epilogue: field -> update (per output element) ----
    const float a_kv = FIELD_ONLY ? 0.0f : __ldg(a_table + k);
    const float lam = FIELD_ONLY ? 0.0f : vqd::pa_lambda(a_kv, a0);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (r >= R) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t c = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            if (c >= n) continue;
            const int64_t p = r * n + c;
            const float F = acc[i][j];
            if (F_out) F_out[p] = F;
            if constexpr (!FIELD_ONLY) {
                float s = S_cur[p], yv = Y[p];
                vqd::step_update(method, F, __ldg(bf + c), a_kv, lam, dt, a0, c0, alpha, s, yv);
                S_nxt[p] = s;
                Y[p] = yv;
            }
        }
    }
}

// F = sum over the k splits (in order), then the update of the step.
template <bool FIELD_ONLY>
__global__ void __launch_bounds__(256) k_dense_finish(int32_t R, int32_t n, int ksplit, const float* __restrict__ part,
                                                      const float* __restrict__ S_cur, float* __restrict__ S_nxt,
                                                      float* __restrict__ Y, const float* __restrict__ bf,
                                                      const float* __restrict__ a_table, int k, float dt, float a0,
                                                      float c0, float* __restrict__ F_out, int method, float alpha) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)R * n;
    if (p >= total) return;
    float F = part[p];
    for (int z = 1; z < ksplit; ++z) F = __fadd_rn(F, part[(int64_t)z * total + p]);
    if (F_out) F_out[p] = F;
    if constexpr (!FIELD_ONLY) {
        const int64_t c = p % n;
        const float a_kv = __ldg(a_table + k);
        float s = S_cur[p], yv = Y[p];
        vqd::step_update(method, F, __ldg(bf + c), a_kv, vqd::pa_lambda(a_kv, a0), dt, a0, c0, alpha, s, yv);
        S_nxt[p] = s;
        Y[p] = yv;
    }
}

// Exact energy of x_r = [S_r > 0] (or of a caller batch of bytes), fixed
// point: parts[g][r] = sum over the 64 rows of tile g of
// x_ri (dfix_i + sum_{j != i} qfix(Q_ij) x_rj), Q as given.
// Block: 32 replicas x 8 row groups; the Q tile is staged in shared memory
// as int64 and broadcast to the 32 replica lanes.
template <typename QT, bool FROM_BYTES>
__global__ void __launch_bounds__(256) k_dense_energy(int64_t R, int32_t n, const QT* __restrict__ Q, int shift,
                                                      const int64_t* __restrict__ dfix, const float* __restrict__ S,
                                                      const uint8_t* __restrict__ X, int64_t* __restrict__ parts) {
    __shared__ int64_t qt[64][33];
    __shared__ uint32_t xw[32];
    __shared__ int64_t red[8][32];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.y * 32 + lane;
    const int64_t i0 = (int64_t)blockIdx.x * 64;
    int64_t row[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) row[q] = 0;
    for (int64_t j0 = 0; j0 < n; j0 += 32) {
        __syncthreads();
        for (int e = threadIdx.x; e < 64 * 32; e += 256) {
            const int ii = e / 32, jj = e % 32;
            const int64_t gi = i0 + ii, gj = j0 + jj;
            qt[ii][jj] = (gi < n && gj < n && gi != gj) ? vqd::qfix<QT>(Q[gi * n + gj], shift) : 0;
        }
        if (g == 0) {
            // bit jj of xw[lane] = x[r][j0 + jj]
            uint32_t w = 0;
            if (r < R)
                for (int jj = 0; jj < 32; ++jj) {
                    const int64_t gj = j0 + jj;
                    bool b = false;
                    if (gj < n) b = FROM_BYTES ? X[r * n + gj] != 0 : S[r * n + gj] > 0.0f;
                    w |= (uint32_t)b << jj;
                }
            xw[lane] = w;
        }
        __syncthreads();
        const uint32_t w = xw[lane];
#pragma unroll 4
        for (int jj = 0; jj < 32; ++jj) {
            const bool on = (w >> jj) & 1u;
#pragma unroll
            for (int q = 0; q < 8; ++q) row[q] += on ? qt[g * 8 + q][jj] : 0;
        }
    }
    int64_t part = 0;
    if (r < R) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t gi = i0 + g * 8 + q;
            if (gi < n) {
                const bool xi = FROM_BYTES ? X[r * n + gi] != 0 : S[r * n + gi] > 0.0f;
                if (xi) part += __ldg(dfix + gi) + row[q];
            }
        }
    }
    red[g][lane] = part;
    __syncthreads();
    if (g == 0 && r < R) {
        int64_t tot = 0;
        for (int q = 0; q < 8; ++q) tot += red[q][lane];
        parts[(int64_t)blockIdx.x * R + r] = tot;
    }
}

// k-splits of the FP32 dense step: enough CTAs to fill the GPU when the
// output tiles alone cannot, with at least 16 k-tiles per split.
void dense_split(int64_t n, int32_t R, int sms, int* ksplit, int* per) {
    const int64_t ctas = div_up(n, BN) * div_up(R, BM);
    const int ktiles = (int)div_up(n, BK);
    int ks = 1;
    if (ctas < sms) ks = (int)std::max<int64_t>(1, std::min<int64_t>(div_up(2 * (int64_t)sms, ctas), ktiles / 16));
    *per = (int)div_up(ktiles, ks);
    *ksplit = (int)div_up(ktiles, *per);
}

template <bool FIELD_ONLY>
int launch_dense_step(veloxq_ctx* ctx, int32_t R, const float* S_cur, float* S_nxt, float* Y, const float* a_table,
                      int k, float dt, float a0, float c0, float* F_out, const Rule& rule) {
    const int32_t n = (int32_t)ctx->n;
    int ksplit, per;
    dense_split(n, R, device_sms(ctx->device), &ksplit, &per);
    float* part = nullptr;
    if (ksplit > 1) {
        // the workspace is sized by dense_prepare before any capture; growing it here is only
        // legal outside a stream capture
        const size_t need = sizeof(float) * (size_t)ksplit * R * n;
        if (ctx->dpart.bytes < need) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            VQ_CUDA(cudaStreamIsCapturing(ctx->stream, &cs));
            if (cs != cudaStreamCaptureStatusNone) return fail(VELOXQ_ECUDA, "dense step workspace not prepared");
            VQ_TRY(ctx->dpart.ensure(need));
        }
        part = ctx->dpart.as<float>();
    }
    dim3 g((unsigned)div_up(n, BN), (unsigned)div_up(R, BM), (unsigned)ksplit);
    // cp.async needs 16-byte aligned rows of Qoff
    const bool async_b = n % 4 == 0 && (reinterpret_cast<uintptr_t>(ctx->qoff32.p) & 15) == 0;
    if (async_b)
        k_dense_step<FIELD_ONLY, true><<<g, 256, 0, ctx->stream>>>(R, n, S_cur, ctx->qoff32.as<float>(), S_nxt, Y,
                                                                   ctx->bf.as<float>(), a_table, k, dt, a0, c0,
                                                                   F_out, rule.method, rule.alpha, per, part);
    else
        k_dense_step<FIELD_ONLY, false><<<g, 256, 0, ctx->stream>>>(R, n, S_cur, ctx->qoff32.as<float>(), S_nxt, Y,
                                                                    ctx->bf.as<float>(), a_table, k, dt, a0, c0,
                                                                    F_out, rule.method, rule.alpha, per, part);
    if (ksplit > 1)
        k_dense_finish<FIELD_ONLY><<<(unsigned)div_up((int64_t)R * n, 256), 256, 0, ctx->stream>>>(
            R, n, ksplit, part, S_cur, S_nxt, Y, ctx->bf.as<float>(), a_table, k, dt, a0, c0, F_out, rule.method,
            rule.alpha);
    VQ_LAUNCH_CHECK("dense_step");
    return VELOXQ_OK;
}

template <bool FROM_BYTES>
int launch_dense_energy(veloxq_ctx* ctx, int64_t R, const float* S, const uint8_t* X, int64_t* parts, int* nparts,
                        bool allow_tc) {
    const int32_t n = (int32_t)ctx->n;
    *nparts = (int)div_up(n, 64);
    if (R == 0) return VELOXQ_OK;
    if (allow_tc && tc_energy_ready(ctx, R)) return tc_energy(ctx, R, S, X, parts, nparts);
    dim3 g((unsigned)div_up(n, 64), (unsigned)div_up(R, 32));
    const int sh = ctx->energy_shift;
    const int64_t* df = ctx->dfix.as<int64_t>();
    switch (ctx->qx_type) {
        case VELOXQ_I8:
            k_dense_energy<int8_t, FROM_BYTES><<<g, 256, 0, ctx->stream>>>(R, n, ctx->qx.as<int8_t>(), sh, df, S, X, parts);
            break;
        case VELOXQ_I32:
            k_dense_energy<int32_t, FROM_BYTES><<<g, 256, 0, ctx->stream>>>(R, n, ctx->qx.as<int32_t>(), sh, df, S, X, parts);
            break;
        case VELOXQ_F32:
            k_dense_energy<float, FROM_BYTES><<<g, 256, 0, ctx->stream>>>(R, n, ctx->qx.as<float>(), sh, df, S, X, parts);
            break;
        case VELOXQ_F64:
            k_dense_energy<double, FROM_BYTES><<<g, 256, 0, ctx->stream>>>(R, n, ctx->qx.as<double>(), sh, df, S, X, parts);
            break;
    }
    VQ_LAUNCH_CHECK("dense_energy");
    return VELOXQ_OK;
}

}  // namespace

int dense_step(veloxq_ctx* ctx, int32_t R, const float* S_cur, float* S_nxt, float* Y, const float* a_table, int k,
               float dt, float a0, float c0, float* F_out, const Rule& rule) {
    return launch_dense_step<false>(ctx, R, S_cur, S_nxt, Y, a_table, k, dt, a0, c0, F_out, rule);
}

int dense_prepare(veloxq_ctx* ctx, int32_t R) {
    int ksplit, per;
    dense_split(ctx->n, R, device_sms(ctx->device), &ksplit, &per);
    if (ksplit > 1) VQ_TRY(ctx->dpart.ensure(sizeof(float) * (size_t)ksplit * R * ctx->n));
    return VELOXQ_OK;
}

int dense_field(veloxq_ctx* ctx, int32_t R, const float* S, float* F) {
    return launch_dense_step<true>(ctx, R, S, nullptr, nullptr, nullptr, 0, 0.f, 0.f, 0.f, F, Rule());
}

// allow_tc: the tensor-core form when tc_energy_prepare has sized it for R
// replicas (the caller then checks ctx->errw)
int dense_energy(veloxq_ctx* ctx, int32_t R, const float* S, int64_t* parts, int* nparts, bool allow_tc) {
    return launch_dense_energy<false>(ctx, R, S, nullptr, parts, nparts, allow_tc);
}

int dense_energy_x(veloxq_ctx* ctx, int64_t B, const uint8_t* X, int64_t* parts, int* nparts, bool allow_tc) {
    return launch_dense_energy<true>(ctx, B, nullptr, X, parts, nparts, allow_tc);
}

}  // namespace vq
