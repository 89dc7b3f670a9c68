// vq_adjoint.cu -- gradient of the mean relaxed energy after K unrolled
// ballistic-SB steps with respect to dt, c0 and the a(t) knots, by a
// hand-written reverse sweep (the adjoint of the step) with checkpointing.
//
// Loss: L = mean_r E_relax(s_K,r), E_relax(s) = s^T Qoff s / 4 + b^T s / 2 + K0
// (the QUBO energy under x = (1 + s)/2, Sec. 2, evaluated at continuous s).
// Step k (App. B, ballistic form), per element:
//   phi = -(F + b)/2, F = Qoff s;  d = -(a0 - a_k) s + c0 phi
//   yh = y + dt d;  sh = s + dt a0 yh;  wall: |sh| > 1 => s' = sign(sh), y' = 0
// Reverse of step k, given g_s', g_y' (gradients w.r.t. s', y'):
//   g_sh = wall ? 0 : g_s'      g_yh = wall ? 0 : g_y'
//   g_s  = g_sh;  g_yh += dt a0 g_sh;          dL/ddt += a0 yh g_sh
//   g_y  = g_yh;  g_s  += -dt (a0 - a_k) g_yh;  g_phi = dt c0 g_yh
//   dL/ddt += d g_yh;  dL/da_k += dt s g_yh;  dL/dc0 += dt phi g_yh
//   g_s  += -Qoff g_phi / 2                      (Qoff symmetric)
// Forward states are kept every C steps; each segment is recomputed forward
// (bit-identical: the same kernels) before its reverse sweep, so the wall
// masks of the reverse sweep are those of the forward run.
#include <cmath>
#include <vector>

#include "vq_internal.cuh"

namespace vq {

namespace {

constexpr int kAdjBlocks = 1216;   // grid-stride; a fixed count fixes the order of the FP64 partial sums
constexpr int kAdjThreads = 256;

template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double* sh /* [N][kAdjThreads] */) {
#pragma unroll
    for (int q = 0; q < N; ++q) sh[q * kAdjThreads + threadIdx.x] = v[q];
    __syncthreads();
    for (int s = kAdjThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int q = 0; q < N; ++q) sh[q * kAdjThreads + threadIdx.x] += sh[q * kAdjThreads + threadIdx.x + s];
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = sh[q * kAdjThreads];
}

// Loss terms and the seed of the reverse sweep: lam_s = (F + b)/(2R), lam_y = 0.
template <int V, typename WT, int UNROLL>
__global__ void __launch_bounds__(kAdjThreads) k_adj_loss(int64_t n, int32_t R, int32_t nvec, const int64_t* __restrict__ rp,
                                                          const int32_t* __restrict__ col, const WT* __restrict__ w,
                                                          float wscale, const float* __restrict__ S,
                                                          const float* __restrict__ bf, float* lam_s, float* lam_y,
                                                          double* parts, int udeg) {
    __shared__ double sh[kAdjThreads];
    double e = 0.0;
    const int64_t total = n * (int64_t)nvec;
    const float invR = 1.0f / (float)R;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i;
        int32_t vi;
        vqd::split_index(t, n, nvec, i, vi);
        const int64_t off = (int64_t)vi * V;
        const int64_t me = i * R + off;
        float acc[V], s[V], ls[V], ly[V];
        vqd::csr_row_dot<V, WT, UNROLL>(rp, col, w, S, R, off, i, acc, udeg);
        vqd::vload<V>(S + me, s);
        const float b = __ldg(bf + i);
#pragma unroll
        for (int l = 0; l < V; ++l) {
            const float F = acc[l] * wscale;
            e += 0.25 * (double)s[l] * (double)F + 0.5 * (double)b * (double)s[l];
            ls[l] = 0.5f * (F + b) * invR;
            ly[l] = 0.0f;
        }
        vqd::vstore<V>(lam_s + me, ls);
        vqd::vstore<V>(lam_y + me, ly);
    }
    double v[1] = {e};
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = v[0];
}

// Reverse of one step, elementwise part (F of s_k recomputed in the forward
// order). Writes the local part of g_s and replaces lam_y by g_y (= g_yh);
// g_phi = dt c0 g_yh is not stored: k_adj_b forms it from the new lam_y
// with the same product, which saves one state array of writes and reads
// per step. Per-block partial sums of (dL/ddt, dL/dc0, dL/da_k).
template <int V, typename WT, int UNROLL>
__global__ void __launch_bounds__(kAdjThreads) k_adj_a(int64_t n, int32_t R, int32_t nvec, const int64_t* __restrict__ rp,
                                                       const int32_t* __restrict__ col, const WT* __restrict__ w,
                                                       float wscale, const float* __restrict__ Sk,
                                                       const float* __restrict__ Yk, const float* __restrict__ bf,
                                                       float a_k, float dt, float a0, float c0,
                                                       const float* __restrict__ lam_s, float* lam_y,
                                                       float* gsl, double* parts3, int udeg) {
    __shared__ double sh[3 * kAdjThreads];
    double acc3[3] = {0.0, 0.0, 0.0};
    const int64_t total = n * (int64_t)nvec;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i;
        int32_t vi;
        vqd::split_index(t, n, nvec, i, vi);
        const int64_t off = (int64_t)vi * V;
        const int64_t me = i * R + off;
        float acc[V], s[V], y[V], ls[V], ly[V], gs[V], gy[V];
        vqd::csr_row_dot<V, WT, UNROLL>(rp, col, w, Sk, R, off, i, acc, udeg);
        vqd::vload<V>(Sk + me, s);
        vqd::vload<V>(Yk + me, y);
        vqd::vload<V>(lam_s + me, ls);
        vqd::vload_plain<V>(lam_y + me, ly);
        const float b = __ldg(bf + i);
        float ddt = 0.0f, dc0 = 0.0f, da = 0.0f;
#pragma unroll
        for (int l = 0; l < V; ++l) {
            const vqd::BsbPre o = vqd::bsb_pre(acc[l] * wscale, b, a_k, dt, a0, c0, s[l], y[l]);
            const bool wall = fabsf(o.sh) > 1.0f;
            const float g_sh = wall ? 0.0f : ls[l];
            float g_yh = wall ? 0.0f : ly[l];
            float g_s = g_sh;
            g_yh += dt * a0 * g_sh;
            ddt += a0 * o.yh * g_sh;
            gy[l] = g_yh;
            g_s += -dt * (a0 - a_k) * g_yh;
            ddt += o.drive * g_yh;
            da += dt * s[l] * g_yh;
            dc0 += dt * o.phi * g_yh;
            gs[l] = g_s;
        }
        vqd::vstore<V>(gsl + me, gs);
        vqd::vstore<V>(lam_y + me, gy);
        acc3[0] += ddt;
        acc3[1] += dc0;
        acc3[2] += da;
    }
    block_sum<3>(acc3, sh);
    if (threadIdx.x == 0) {
        parts3[3 * blockIdx.x + 0] = acc3[0];
        parts3[3 * blockIdx.x + 1] = acc3[1];
        parts3[3 * blockIdx.x + 2] = acc3[2];
    }
}

// lam_s = g_s(local) - Qoff g_phi / 2, with g_phi_j = dt c0 g_y_j formed
// from the gathered g_y (the new lam_y) as k_adj_a would have formed it.
// The six-at-once gather of lattices fits 32 registers, eight blocks per SM
// (0.54 against 0.65 ms at 34 registers and seven blocks, lattice L = 100,
// 256 replicas); the four-at-a-time forms would spill there and keep their
// own count.
template <int V, typename WT, int UNROLL>
__global__ void __launch_bounds__(kAdjThreads, UNROLL == 6 ? 8 : 1) k_adj_b(int64_t n, int32_t R, int32_t nvec, const int64_t* __restrict__ rp,
                                                       const int32_t* __restrict__ col, const WT* __restrict__ w,
                                                       float wscale, const float* __restrict__ gy, float dt, float c0,
                                                       const float* __restrict__ gsl, float* lam_s, int udeg) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * nvec) return;
    int64_t i;
    int32_t vi;
    vqd::split_index(t, n, nvec, i, vi);
    const int64_t off = (int64_t)vi * V;
    const int64_t me = i * R + off;
    float acc[V], g[V];
    vqd::csr_row_dot<V, WT, UNROLL, false, true>(rp, col, w, gy, R, off, i, acc, udeg, dt * c0);
    vqd::vload<V>(gsl + me, g);
#pragma unroll
    for (int l = 0; l < V; ++l) g[l] = g[l] - 0.5f * (acc[l] * wscale);
    vqd::vstore<V>(lam_s + me, g);
}

// acc[0] += dL/ddt, acc[1] += dL/dc0, acc[2 + k] = dL/da_k (fixed order)
__global__ void k_adj_reduce(const double* __restrict__ parts3, int G, int k, double* acc) {
    __shared__ double sh[3 * kAdjThreads];
    double v[3] = {0.0, 0.0, 0.0};
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        v[0] += parts3[3 * g];
        v[1] += parts3[3 * g + 1];
        v[2] += parts3[3 * g + 2];
    }
    block_sum<3>(v, sh);
    if (threadIdx.x == 0) {
        acc[0] += v[0];
        acc[1] += v[1];
        acc[2 + k] = v[2];
    }
}

__global__ void k_adj_loss_total(const double* __restrict__ parts, int G, double* out) {
    __shared__ double sh[kAdjThreads];
    double v[1] = {0.0};
    for (int g = threadIdx.x; g < G; g += blockDim.x) v[0] += parts[g];
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) *out = v[0];
}

// dL/dknot_j = sum_k w_kj dL/da_k, with the interpolation weights of the schedule.
__global__ void k_adj_knots(int K, int nk, const double* __restrict__ da, double* dknots) {
    const int j = threadIdx.x;
    if (j >= nk) return;
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
        double wj;
        if (K == 1 || nk == 1) wj = (j == 0) ? 1.0 : 0.0;
        else {
            const double t = (double)k * (double)(nk - 1) / (double)(K - 1);
            int lo = (int)floor(t);
            if (lo > nk - 2) lo = nk - 2;
            const double f = t - (double)lo;
            wj = (j == lo) ? 1.0 - f : (j == lo + 1) ? f : 0.0;
        }
        s += wj * da[k];
    }
    dknots[j] = s;
}

// The reverse sweep recomputes F with the gather variant the forward used,
// so the wall masks agree bit for bit.
template <int V, typename WT, int U>
struct AdjLaunch {
    static void loss(veloxq_ctx* c, int32_t R, const WT* w, float ws, const float* S, float* ls, float* ly, double* parts) {
        k_adj_loss<V, WT, U><<<kAdjBlocks, kAdjThreads, 0, c->stream>>>(c->n, R, R / V, c->rowptr.as<int64_t>(),
                                                                         c->col.as<int32_t>(), w, ws, S,
                                                                         c->bf.as<float>(), ls, ly, parts, c->uniform_deg);
    }
    static void a(veloxq_ctx* c, int32_t R, const WT* w, float ws, const float* Sk, const float* Yk, float a_k, float dt,
                  float a0, float c0, const float* ls, float* ly, float* gs, double* parts3) {
        k_adj_a<V, WT, U><<<kAdjBlocks, kAdjThreads, 0, c->stream>>>(c->n, R, R / V, c->rowptr.as<int64_t>(),
                                                                      c->col.as<int32_t>(), w, ws, Sk, Yk,
                                                                      c->bf.as<float>(), a_k, dt, a0, c0, ls, ly, gs,
                                                                      parts3, c->uniform_deg);
    }
    static void b(veloxq_ctx* c, int32_t R, const WT* w, float ws, const float* gy, float dt, float c0, const float* gs,
                  float* ls) {
        const int64_t total = c->n * (int64_t)(R / V);
        k_adj_b<V, WT, U><<<(unsigned)div_up(total, kAdjThreads), kAdjThreads, 0, c->stream>>>(
            c->n, R, R / V, c->rowptr.as<int64_t>(), c->col.as<int32_t>(), w, ws, gy, dt, c0, gs, ls, c->uniform_deg);
    }
};

template <typename WT, int U>
void adj_loss_v(veloxq_ctx* c, int V, int32_t R, const WT* w, float ws, const float* S, float* ls, float* ly,
                double* parts) {
    if (V == 4) AdjLaunch<4, WT, U>::loss(c, R, w, ws, S, ls, ly, parts);
    else if (V == 2) AdjLaunch<2, WT, U>::loss(c, R, w, ws, S, ls, ly, parts);
    else AdjLaunch<1, WT, U>::loss(c, R, w, ws, S, ls, ly, parts);
}
template <typename WT, int U>
void adj_step_v(veloxq_ctx* c, int V, int32_t R, const WT* w, float ws, const float* Sk, const float* Yk, float a_k,
                float dt, float a0, float c0, float* ls, float* ly, float* gs, double* parts3) {
    if (V == 4) AdjLaunch<4, WT, U>::a(c, R, w, ws, Sk, Yk, a_k, dt, a0, c0, ls, ly, gs, parts3);
    else if (V == 2) AdjLaunch<2, WT, U>::a(c, R, w, ws, Sk, Yk, a_k, dt, a0, c0, ls, ly, gs, parts3);
    else AdjLaunch<1, WT, U>::a(c, R, w, ws, Sk, Yk, a_k, dt, a0, c0, ls, ly, gs, parts3);
    if (V == 4) AdjLaunch<4, WT, U>::b(c, R, w, ws, ly, dt, c0, gs, ls);
    else if (V == 2) AdjLaunch<2, WT, U>::b(c, R, w, ws, ly, dt, c0, gs, ls);
    else AdjLaunch<1, WT, U>::b(c, R, w, ws, ly, dt, c0, gs, ls);
}

template <typename WT>
int adj_dispatch_loss(veloxq_ctx* c, int V, int32_t R, const WT* w, float ws, const float* S, float* ls, float* ly,
                      double* parts) {
    if (c->stream_unroll == 6 && c->uniform_deg == 6) adj_loss_v<WT, 6>(c, V, R, w, ws, S, ls, ly, parts);
    else if (c->stream_unroll == 4) adj_loss_v<WT, 4>(c, V, R, w, ws, S, ls, ly, parts);
    else adj_loss_v<WT, 1>(c, V, R, w, ws, S, ls, ly, parts);
    VQ_LAUNCH_CHECK("adjoint loss");
    return VELOXQ_OK;
}
template <typename WT>
int adj_dispatch_step(veloxq_ctx* c, int V, int32_t R, const WT* w, float ws, const float* Sk, const float* Yk, float a_k,
                      float dt, float a0, float c0, float* ls, float* ly, float* gs, double* parts3) {
    if (c->stream_unroll == 6 && c->uniform_deg == 6)
        adj_step_v<WT, 6>(c, V, R, w, ws, Sk, Yk, a_k, dt, a0, c0, ls, ly, gs, parts3);
    else if (c->stream_unroll == 4) adj_step_v<WT, 4>(c, V, R, w, ws, Sk, Yk, a_k, dt, a0, c0, ls, ly, gs, parts3);
    else adj_step_v<WT, 1>(c, V, R, w, ws, Sk, Yk, a_k, dt, a0, c0, ls, ly, gs, parts3);
    VQ_LAUNCH_CHECK("adjoint step");
    return VELOXQ_OK;
}

}  // namespace

// Checkpointed forward + reverse sweep on the streaming sparse path.
// a_table (device) holds a_k; a_host the same values on the host.
int adjoint_run(veloxq_ctx* ctx, int32_t R, const RunParams& p, const std::vector<float>& a_host, uint64_t seed,
                int32_t C, double* loss, double* d_dt, double* d_c0, double* d_knots, int n_knots, AdjTiming* tm) {
    const int64_t n = ctx->n, nR = n * (int64_t)R;
    const int K = p.K;
    const int M = (int)div_up(K, C);                  // checkpoints: states before steps 0, C, 2C, ...
    const int V = vec_width(R);
    const size_t blk = sizeof(float) * (size_t)nR;
    // checkpoints (S, Y) x M, segment states (S, Y) x C, 3 adjoint blocks
    DevBuf ck, seg, adj, red;
    VQ_TRY(ck.ensure(2 * blk * (size_t)M));
    VQ_TRY(seg.ensure(2 * blk * (size_t)(C + 1)));
    VQ_TRY(adj.ensure(3 * blk));
    VQ_TRY(red.ensure(sizeof(double) * (size_t)(3 * kAdjBlocks + kAdjBlocks + 2 + K + 8 + n_knots)));
    auto ckS = [&](int m) { return ck.as<float>() + (size_t)(2 * m) * nR; };
    auto ckY = [&](int m) { return ck.as<float>() + (size_t)(2 * m + 1) * nR; };
    auto sgS = [&](int t) { return seg.as<float>() + (size_t)(2 * t) * nR; };
    auto sgY = [&](int t) { return seg.as<float>() + (size_t)(2 * t + 1) * nR; };
    float* lam_s = adj.as<float>();
    float* lam_y = lam_s + nR;
    float* gsl = lam_y + nR;
    double* parts3 = red.as<double>();
    double* parts = parts3 + 3 * kAdjBlocks;
    double* acc = parts + kAdjBlocks;                  // [0] ddt [1] dc0 [2..2+K) da_k
    double* lossd = acc + 2 + K;
    double* dkn = lossd + 8;
    const float* at = ctx->a_table.as<float>();
    cudaStream_t st = ctx->stream;
    // events: [0] start, [1] end, then (before, after) each segment's reverse steps
    struct Events {
        std::vector<cudaEvent_t> e;
        ~Events() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    ev.e.assign((size_t)(2 + 2 * M), nullptr);
    for (cudaEvent_t& x : ev.e) VQ_CUDA(cudaEventCreate(&x));
    VQ_CUDA(cudaEventRecord(ev.e[0], st));
    int64_t launches = 0;
    VQ_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)(2 + K), st));

    // ---- forward with checkpoints (two working buffers in seg[0], seg[1]) ----
    VQ_TRY(launch_init_state(ctx, R, seed, p.sigma0, LAYOUT_NR, sgS(0), sgY(0)));
    float* cS = sgS(0);
    float* cY = sgY(0);
    float* nS = sgS(1);
    for (int k = 0; k < K; ++k) {
        if (k % C == 0) {
            VQ_CUDA(cudaMemcpyAsync(ckS(k / C), cS, blk, cudaMemcpyDeviceToDevice, st));
            VQ_CUDA(cudaMemcpyAsync(ckY(k / C), cY, blk, cudaMemcpyDeviceToDevice, st));
        }
        VQ_TRY(stream_step_y(ctx, R, cS, nS, cY, cY, at, k, p.dt, p.a0, p.c0, nullptr));
        std::swap(cS, nS);
    }
    launches += 1 + K + 2;   // init, forward steps, loss and its total
    // ---- loss and seed ----
    if (ctx->w8.p) VQ_TRY(adj_dispatch_loss<int8_t>(ctx, V, R, ctx->w8.as<int8_t>(), 0.5f, cS, lam_s, lam_y, parts));
    else VQ_TRY(adj_dispatch_loss<float>(ctx, V, R, ctx->wf.as<float>(), 1.0f, cS, lam_s, lam_y, parts));
    k_adj_loss_total<<<1, kAdjThreads, 0, st>>>(parts, kAdjBlocks, lossd);
    VQ_LAUNCH_CHECK("adjoint loss total");

    // ---- reverse sweep, one segment at a time ----
    for (int m = M - 1; m >= 0; --m) {
        const int k0 = m * C, k1 = std::min(K, k0 + C);
        // recompute the segment: state t (before step k0 + t) into seg[t]
        VQ_CUDA(cudaMemcpyAsync(sgS(0), ckS(m), blk, cudaMemcpyDeviceToDevice, st));
        VQ_CUDA(cudaMemcpyAsync(sgY(0), ckY(m), blk, cudaMemcpyDeviceToDevice, st));
        for (int t = 0; t < k1 - k0 - 1; ++t)
            VQ_TRY(stream_step_y(ctx, R, sgS(t), sgS(t + 1), sgY(t), sgY(t + 1), at, k0 + t, p.dt, p.a0, p.c0, nullptr));
        launches += k1 - k0 - 1 + 3 * (k1 - k0);
        VQ_CUDA(cudaEventRecord(ev.e[2 + 2 * m], st));
        for (int k = k1 - 1; k >= k0; --k) {
            const int t = k - k0;
            if (ctx->w8.p)
                VQ_TRY(adj_dispatch_step<int8_t>(ctx, V, R, ctx->w8.as<int8_t>(), 0.5f, sgS(t), sgY(t), a_host[k], p.dt,
                                                 p.a0, p.c0, lam_s, lam_y, gsl, parts3));
            else
                VQ_TRY(adj_dispatch_step<float>(ctx, V, R, ctx->wf.as<float>(), 1.0f, sgS(t), sgY(t), a_host[k], p.dt,
                                                p.a0, p.c0, lam_s, lam_y, gsl, parts3));
            k_adj_reduce<<<1, kAdjThreads, 0, st>>>(parts3, kAdjBlocks, k, acc);
            VQ_LAUNCH_CHECK("adjoint reduce");
        }
        VQ_CUDA(cudaEventRecord(ev.e[3 + 2 * m], st));
    }
    k_adj_knots<<<1, 64, 0, st>>>(K, n_knots, acc + 2, dkn);
    VQ_LAUNCH_CHECK("adjoint knots");
    launches += 1;
    VQ_CUDA(cudaEventRecord(ev.e[1], st));
    std::vector<double> h((size_t)(2 + K + 8 + n_knots));
    VQ_CUDA(cudaMemcpyAsync(h.data(), acc, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
    VQ_CUDA(cudaStreamSynchronize(st));
    if (tm) {
        VQ_CUDA(cudaEventElapsedTime(&tm->ms_total, ev.e[0], ev.e[1]));
        tm->ms_reverse = 0.f;
        for (int m = 0; m < M; ++m) {
            float x = 0.f;
            VQ_CUDA(cudaEventElapsedTime(&x, ev.e[2 + 2 * m], ev.e[3 + 2 * m]));
            tm->ms_reverse += x;
        }
        tm->launches = launches;
        tm->reverse_launches = 3 * (int64_t)K;
    }
    if (loss) *loss = ctx->K0 + h[2 + K] / (double)R;
    if (d_dt) *d_dt = h[0];
    if (d_c0) *d_c0 = h[1];
    if (d_knots)
        for (int j = 0; j < n_knots; ++j) d_knots[j] = h[2 + K + 8 + j];
    return VELOXQ_OK;
}

}  // namespace vq
