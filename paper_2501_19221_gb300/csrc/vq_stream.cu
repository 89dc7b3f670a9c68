// vq_stream.cu -- sparse local field fused with the ballistic-SB update, one
// launch per step, state in HBM (variable-major [n][R]: the R replicas of a
// variable are contiguous, so a neighbour's state is one coalesced vector
// load shared by all lanes of the row), plus the exact readout energy.
//
// Step (App. B, ballistic form):  F_i = sum_{j != i} Qs_ij s_j  over the CSR
// row of i, then phi, y, s, walls. Couplings come as FP32 Qs or, for integer
// instances with |2 Qs| <= 127, as int8 2Qs (F = acc / 2, exact scaling).
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "vq_internal.cuh"

namespace vq {

namespace {

using vqd::vload;
using vqd::vload_plain;
using vqd::vload_stream;
using vqd::vstore_stream;
using vqd::vstore;
using vqd::wval;

// One thread per (variable i, vector v of V replicas). Y_in and Y_out may be
// the same buffer (in-place update). SIGN: the field is of PA's binarised
// spins; method selects the update (veloxq_method).
template <int V, typename WT, bool FIELD_ONLY, int UNROLL, bool SIGN>
__global__ void __launch_bounds__(256) k_stream_step(int64_t n, int32_t R, int32_t nvec, const int64_t* __restrict__ rp,
                                                     const int32_t* __restrict__ col, const WT* __restrict__ w,
                                                     float wscale, const float* __restrict__ S_cur,
                                                     float* __restrict__ S_nxt, const float* Y_in, float* Y_out,
                                                     const float* __restrict__ bf, const float* __restrict__ a_table,
                                                     int k, float dt, float a0, float c0, float* __restrict__ F_out,
                                                     int udeg, int method, float alpha, int32_t cvec) {
    // threads in chunk-major order: all rows of replica vectors [c cvec,
    // (c+1) cvec) before the next chunk (cvec = nvec: one chunk), so that
    // the neighbours' states a wave gathers span one chunk of every row
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * nvec) return;
    int64_t i;
    int32_t v;
    if (cvec == nvec) {
        vqd::split_index(t, n, nvec, i, v);
    } else {
        // chunk c = t / (n cvec), then row and vector within the chunk
        int64_t c, rem;
        if (n * nvec < (int64_t(1) << 32)) {
            const uint32_t per_chunk = (uint32_t)n * (uint32_t)cvec;
            c = (uint32_t)t / per_chunk;
            rem = t - c * per_chunk;
        } else {
            c = t / (n * cvec);
            rem = t - c * n * cvec;
        }
        int32_t w;
        vqd::split_index(rem, n, cvec, i, w);
        v = (int32_t)(c * cvec) + w;
    }
    const int64_t off = (int64_t)v * V;
    const int64_t me = i * R + off;
    // the variable's own state first: independent of the couplings, in flight during the gathers
    float s[V], y[V], b = 0.0f, a_k = 0.0f;
    if constexpr (!FIELD_ONLY) {
        vload<V>(S_cur + me, s);
        vload_stream<V>(Y_in + me, y);
        b = __ldg(bf + i);
        a_k = __ldg(a_table + k);
    }
    float acc[V];
    vqd::csr_row_dot<V, WT, UNROLL, SIGN>(rp, col, w, S_cur, R, off, i, acc, udeg);
    float F[V];
#pragma unroll
    for (int l = 0; l < V; ++l) F[l] = acc[l] * wscale;     // wscale is 1 or 1/2: exact
    if (F_out) vstore<V>(F_out + me, F);
    if constexpr (FIELD_ONLY) return;
    if (method == vqd::METHOD_BSB) {
#pragma unroll
        for (int l = 0; l < V; ++l) vqd::bsb_update(F[l], b, a_k, dt, a0, c0, s[l], y[l]);
    } else {
        const float lam = vqd::pa_lambda(a_k, a0);
#pragma unroll
        for (int l = 0; l < V; ++l) vqd::step_update(method, F[l], b, a_k, lam, dt, a0, c0, alpha, s[l], y[l]);
    }
    vstore_stream<V>(S_nxt + me, s);
    vstore_stream<V>(Y_out + me, y);
}

__device__ __forceinline__ int64_t ewval(int8_t w) { return (int64_t)w; }
__device__ __forceinline__ int64_t ewval(int64_t w) { return w; }

// Exact readout energy, fixed point: parts[g][r] = sum over the rows of group
// g of x_ri (dfix_i + sum_j wE_ij x_rj), x = [s > 0]. Block (TX, TY): TX
// vectors of replicas, TY rows; rows of a group are grid-strided.
template <int V, typename EW>
__global__ void __launch_bounds__(256) k_stream_energy(int64_t n, int32_t R, int32_t nvec, const int64_t* __restrict__ rp,
                                                       const int32_t* __restrict__ col, const EW* __restrict__ we,
                                                       const int64_t* __restrict__ dfix, const float* __restrict__ S,
                                                       int64_t* __restrict__ parts) {
    extern __shared__ int64_t sh[];
    const int TX = blockDim.x, TY = blockDim.y;
    const int32_t v = blockIdx.x * TX + threadIdx.x;
    int64_t part[V];
#pragma unroll
    for (int l = 0; l < V; ++l) part[l] = 0;
    if (v < nvec) {
        const int64_t off = (int64_t)v * V;
        for (int64_t i = (int64_t)blockIdx.y * TY + threadIdx.y; i < n; i += (int64_t)gridDim.y * TY) {
            float si[V];
            vload<V>(S + i * R + off, si);
            bool any = false;
#pragma unroll
            for (int l = 0; l < V; ++l) any |= si[l] > 0.0f;
            if (!any) continue;
            int64_t row[V];
#pragma unroll
            for (int l = 0; l < V; ++l) row[l] = 0;
            const int64_t p1 = __ldg(rp + i + 1);
            for (int64_t p = __ldg(rp + i); p < p1; ++p) {
                const int64_t j = __ldg(col + p);
                const int64_t wq = ewval(__ldg(we + p));
                float sj[V];
                vload<V>(S + j * R + off, sj);
#pragma unroll
                for (int l = 0; l < V; ++l) row[l] += sj[l] > 0.0f ? wq : 0;
            }
            const int64_t d = __ldg(dfix + i);
#pragma unroll
            for (int l = 0; l < V; ++l) part[l] += si[l] > 0.0f ? d + row[l] : 0;
        }
    }
    // reduce over TY in a fixed order
#pragma unroll
    for (int l = 0; l < V; ++l) sh[((int64_t)threadIdx.y * TX + threadIdx.x) * V + l] = part[l];
    __syncthreads();
    if (threadIdx.y == 0 && v < nvec) {
#pragma unroll
        for (int l = 0; l < V; ++l) {
            int64_t tot = 0;
            for (int y = 0; y < TY; ++y) tot += sh[((int64_t)y * TX + threadIdx.x) * V + l];
            const int32_t r = v * V + l;
            if (r < R) parts[(int64_t)blockIdx.y * R + r] = tot;
        }
    }
}

// Energy of a caller batch X [B][n] (uint8): parts[g][b].
template <typename EW>
__global__ void __launch_bounds__(256) k_sparse_energy_x(int64_t n, int64_t B, const int64_t* __restrict__ rp,
                                                         const int32_t* __restrict__ col, const EW* __restrict__ we,
                                                         const int64_t* __restrict__ dfix, const uint8_t* __restrict__ X,
                                                         int64_t* __restrict__ parts) {
    __shared__ int64_t sh[256];
    const int64_t b = blockIdx.y;
    const uint8_t* x = X + b * n;
    int64_t part = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!x[i]) continue;
        int64_t row = __ldg(dfix + i);
        const int64_t p1 = __ldg(rp + i + 1);
        for (int64_t p = __ldg(rp + i); p < p1; ++p)
            if (x[__ldg(col + p)]) row += ewval(__ldg(we + p));
        part += row;
    }
    sh[threadIdx.x] = part;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[(int64_t)blockIdx.x * B + b] = sh[0];
}

template <bool FIELD_ONLY, bool SIGN>
int launch_step(veloxq_ctx* ctx, int32_t R, const float* S_cur, float* S_nxt, const float* Y_in, float* Y_out,
                const float* a_table, int k, float dt, float a0, float c0, float* F_out, const Rule& rule) {
    const int V = vec_width(R);
    const int32_t nvec = R / V;
    const int32_t cvec = (ctx->stream_cvec > 0 && nvec % ctx->stream_cvec == 0) ? ctx->stream_cvec : nvec;
    const int64_t total = ctx->n * (int64_t)nvec;
    const unsigned g = (unsigned)div_up(total, 256);
    const int64_t* rp = ctx->rowptr.as<int64_t>();
    const int32_t* cl = ctx->col.as<int32_t>();
    const float* bf = ctx->bf.as<float>();
    cudaStream_t st = ctx->stream;
#define VQ_STEP_U(VV, WT, WPTR, SC, U)                                                                       \
    k_stream_step<VV, WT, FIELD_ONLY, U, SIGN><<<g, 256, 0, st>>>(ctx->n, R, nvec, rp, cl, WPTR, SC, S_cur, S_nxt, \
                                                                  Y_in, Y_out, bf, a_table, k, dt, a0, c0, F_out, \
                                                                  ctx->uniform_deg, rule.method, rule.alpha, cvec)
#define VQ_STEP(VV, WT, WPTR, SC)                                   \
    do {                                                            \
        if (unroll == 6) VQ_STEP_U(VV, WT, WPTR, SC, 6);            \
        else if (unroll == 4) VQ_STEP_U(VV, WT, WPTR, SC, 4);       \
        else VQ_STEP_U(VV, WT, WPTR, SC, 1);                        \
    } while (0)
    const int unroll = (ctx->stream_unroll == 6 && ctx->uniform_deg == 6) ? 6 : ctx->stream_unroll == 4 ? 4 : 1;
    if (ctx->w8.p) {
        const int8_t* w = ctx->w8.as<int8_t>();
        if (V == 4) VQ_STEP(4, int8_t, w, 0.5f); else if (V == 2) VQ_STEP(2, int8_t, w, 0.5f); else VQ_STEP(1, int8_t, w, 0.5f);
    } else {
        const float* w = ctx->wf.as<float>();
        if (V == 4) VQ_STEP(4, float, w, 1.0f); else if (V == 2) VQ_STEP(2, float, w, 1.0f); else VQ_STEP(1, float, w, 1.0f);
    }
#undef VQ_STEP
#undef VQ_STEP_U
    VQ_LAUNCH_CHECK("stream_step");
    return VELOXQ_OK;
}

}  // namespace

int vec_width(int32_t R) { return (R % 4 == 0) ? 4 : (R % 2 == 0) ? 2 : 1; }

int stream_step(veloxq_ctx* ctx, int32_t R, const float* S_cur, float* S_nxt, float* Y, const float* a_table, int k,
                float dt, float a0, float c0, float* F_out, const Rule& rule) {
    if (rule.method == VELOXQ_METHOD_PA)
        return launch_step<false, true>(ctx, R, S_cur, S_nxt, Y, Y, a_table, k, dt, a0, c0, F_out, rule);
    return launch_step<false, false>(ctx, R, S_cur, S_nxt, Y, Y, a_table, k, dt, a0, c0, F_out, rule);
}

int stream_step_y(veloxq_ctx* ctx, int32_t R, const float* S_cur, float* S_nxt, const float* Y_in, float* Y_out,
                  const float* a_table, int k, float dt, float a0, float c0, float* F_out, const Rule& rule) {
    if (rule.method == VELOXQ_METHOD_PA)
        return launch_step<false, true>(ctx, R, S_cur, S_nxt, Y_in, Y_out, a_table, k, dt, a0, c0, F_out, rule);
    return launch_step<false, false>(ctx, R, S_cur, S_nxt, Y_in, Y_out, a_table, k, dt, a0, c0, F_out, rule);
}

int stream_field(veloxq_ctx* ctx, int32_t R, const float* S, float* F) {
    return launch_step<true, false>(ctx, R, S, nullptr, nullptr, nullptr, nullptr, 0, 0.f, 0.f, 0.f, F, Rule());
}

// Chunk widths (replica vectors) worth trying for R replicas: when one state
// array is larger than about half of L2, the widths whose chunk of every row
// (n x width x V floats) fits in 64 MB, at least 32 replicas (one 128-byte
// line per row) and dividing the vectors of a row; 0 (no chunking) always.
static std::vector<int32_t> chunk_candidates(int64_t n, int32_t R) {
    const int V = vec_width(R);
    const int32_t nvec = R / V;
    const int64_t budget = int64_t(64) << 20;
    std::vector<int32_t> out = {0};
    if (n * (int64_t)R * 4 <= budget) return out;
    int32_t widest = 0;
    for (int32_t cv = nvec / 2; cv * V >= 32; --cv)
        if (nvec % cv == 0 && n * (int64_t)cv * V * 4 <= budget) {
            widest = cv;
            break;
        }
    if (widest) {
        out.push_back(widest);
        for (int32_t cv = widest / 2; cv * V >= 32; --cv)
            if (nvec % cv == 0) {
                out.push_back(cv);
                break;
            }
    }
    return out;
}

// Pick the gather variant (one, four or six couplings at a time) and the
// replica chunk width of the streaming kernels for R replicas by timing steps
// of each pair on the caller's buffers (contents are overwritten);
// VELOXQ_STREAM_FORM fixes them instead.
// Runs eagerly on ctx->stream; must not be called during stream capture.
int stream_autotune(veloxq_ctx* ctx, int32_t R, float* S_a, float* S_b, float* Y) {
    if (ctx->stream_unroll != 0 && ctx->stream_tuned_R == R) return VELOXQ_OK;
    if (const char* form = std::getenv("VELOXQ_STREAM_FORM")) {
        // a form fixed by the caller: "gather chunk", the chunk in replicas (0: all at once)
        const int V = vec_width(R);
        const int32_t nvec = R / V;
        int u = 0, cr = -1;
        const bool parsed = std::sscanf(form, "%d %d", &u, &cr) == 2 && cr >= 0 && cr % V == 0;
        const int32_t cv = parsed ? cr / V : -1;
        const bool ok = parsed && (u == 1 || u == 4 || (u == 6 && ctx->uniform_deg == 6)) &&
                        (cv == 0 || nvec % cv == 0);
        if (!ok)
            return fail(VELOXQ_EINVAL, "VELOXQ_STREAM_FORM must be \"gather chunk\": gather 1, 4 or 6 (rows of exactly "
                                       "6 couplings) and a chunk of replicas (0: all) that the replica count splits "
                                       "into");
        ctx->stream_unroll = u;
        ctx->stream_cvec = cv;
        ctx->stream_tuned_R = R;
        return VELOXQ_OK;
    }
    cudaEvent_t e0, e1;
    VQ_CUDA(cudaEventCreate(&e0));
    VQ_CUDA(cudaEventCreate(&e1));
    VQ_TRY(launch_init_state(ctx, R, 1, 0.1f, LAYOUT_NR, S_a, Y));
    const float* at = ctx->a_table.as<float>();
    std::vector<std::pair<int, int32_t>> cands;   // (gather, chunk)
    for (int32_t cv : chunk_candidates(ctx->n, R))
        for (int u : {1, 4, 6})
            if (u != 6 || ctx->uniform_deg == 6) cands.emplace_back(u, cv);
    auto timed = [&](int reps, float* ms) -> int {
        VQ_CUDA(cudaEventRecord(e0, ctx->stream));
        for (int k = 0; k < reps; ++k)
            VQ_TRY((launch_step<false, false>(ctx, R, (k & 1) ? S_b : S_a, (k & 1) ? S_a : S_b, Y, Y, at, 0, 0.5f,
                                              1.0f, 0.1f, nullptr, Rule())));
        VQ_CUDA(cudaEventRecord(e1, ctx->stream));
        VQ_CUDA(cudaEventSynchronize(e1));
        VQ_CUDA(cudaEventElapsedTime(ms, e0, e1));
        return VELOXQ_OK;
    };
    // Two rounds over all candidates, each timing `reps` steps of one form
    // (10 when a step is shorter than 0.3 ms, else 3); a form's time is its
    // faster round, so a round disturbed by the previous form's state in L2
    // or by a clock change does not decide the pick.
    std::vector<float> per_step(cands.size(), 1e30f);
    int reps = 3;
    for (int round = 0; round < 2; ++round)
        for (size_t c = 0; c < cands.size(); ++c) {
            ctx->stream_unroll = cands[c].first;
            ctx->stream_cvec = cands[c].second;
            float ms = 0.f;
            if (round == 0) {
                VQ_TRY(timed(1, &ms));                 // warm; the first form's step sets the step count
                if (c == 0 && ms < 0.3f) reps = 10;
            }
            VQ_TRY(timed(reps, &ms));
            per_step[c] = std::min(per_step[c], ms / (float)reps);
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    size_t bi = 0;
    for (size_t c = 1; c < cands.size(); ++c)
        if (per_step[c] < per_step[bi]) bi = c;
    const int pick = cands[bi].first;
    const int32_t pick_cv = cands[bi].second;
    ctx->stream_unroll = pick;
    ctx->stream_cvec = pick_cv;
    ctx->stream_tuned_R = R;
    return VELOXQ_OK;
}

// number of row groups (partial sums) used by stream_energy
static int energy_groups(int32_t gx) { return std::max(1, 608 / std::max(1, gx)); }

int stream_energy(veloxq_ctx* ctx, int32_t R, const float* S, int64_t* parts, int* nparts) {
    const int V = vec_width(R);
    const int32_t nvec = R / V;
    int TX = 1;
    while (TX < nvec && TX < 32) TX <<= 1;
    const int TY = 256 / TX;
    const int32_t gx = (int32_t)div_up(nvec, TX);
    const int gy = energy_groups(gx);
    *nparts = gy;
    dim3 blk(TX, TY), grd(gx, gy);
    const size_t sm = sizeof(int64_t) * 256 * V;
    cudaStream_t st = ctx->stream;
    const int64_t* rp = ctx->rowptr.as<int64_t>();
    const int32_t* cl = ctx->col.as<int32_t>();
    const int64_t* df = ctx->dfix.as<int64_t>();
#define VQ_EN(VV, EW, WPTR) k_stream_energy<VV, EW><<<grd, blk, sm, st>>>(ctx->n, R, nvec, rp, cl, WPTR, df, S, parts)
    if (ctx->w8.p) {
        const int8_t* w = ctx->w8.as<int8_t>();
        if (V == 4) VQ_EN(4, int8_t, w); else if (V == 2) VQ_EN(2, int8_t, w); else VQ_EN(1, int8_t, w);
    } else {
        const int64_t* w = ctx->wfix.as<int64_t>();
        if (V == 4) VQ_EN(4, int64_t, w); else if (V == 2) VQ_EN(2, int64_t, w); else VQ_EN(1, int64_t, w);
    }
#undef VQ_EN
    VQ_LAUNCH_CHECK("stream_energy");
    return VELOXQ_OK;
}

int stream_energy_parts(int32_t R) {
    const int V = vec_width(R);
    const int32_t nvec = R / V;
    int TX = 1;
    while (TX < nvec && TX < 32) TX <<= 1;
    return energy_groups((int32_t)div_up(nvec, TX));
}

int sparse_energy_x(veloxq_ctx* ctx, int64_t B, const uint8_t* X, int64_t* parts, int* nparts) {
    const int G = 64;
    *nparts = G;
    if (B == 0) return VELOXQ_OK;
    dim3 grd(G, (unsigned)B);
    if (ctx->w8.p)
        k_sparse_energy_x<int8_t><<<grd, 256, 0, ctx->stream>>>(ctx->n, B, ctx->rowptr.as<int64_t>(), ctx->col.as<int32_t>(),
                                                                ctx->w8.as<int8_t>(), ctx->dfix.as<int64_t>(), X, parts);
    else
        k_sparse_energy_x<int64_t><<<grd, 256, 0, ctx->stream>>>(ctx->n, B, ctx->rowptr.as<int64_t>(), ctx->col.as<int32_t>(),
                                                                 ctx->wfix.as<int64_t>(), ctx->dfix.as<int64_t>(), X, parts);
    VQ_LAUNCH_CHECK("sparse_energy_x");
    return VELOXQ_OK;
}

}  // namespace vq
