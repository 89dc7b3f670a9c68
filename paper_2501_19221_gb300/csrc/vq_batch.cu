// vq_batch.cu -- many dense instances of uneven size in ONE persistent launch
// (BF16 tensor-core field, FP32 state, fused ballistic-SB update).
//
// Each CTA owns a list of whole instances (no synchronisation between CTAs);
// the host assigns instances to CTAs longest-first (LPT on n^2). For each
// instance and step, the CTA walks its 128-row tiles: warp 0 streams the
// pre-tiled operands with 1-D bulk copies, warp 1 issues the MMAs
// (M = 128 variables, N = R replicas, K = variables) into one of two tensor
// memory buffers, warps 2-5 read the other buffer back and update their rows
// (the epilogue of tile t overlaps the main loop of tile t + 1). After the
// last tile of a step the epilogue warps publish the next operand (a proxy
// fence and a named barrier) before the producer may read it.
//
// Operand layout in global memory (the layout the MMA reads from shared
// memory, so that a plain bulk copy lands it there): 128-byte rows, 16-byte
// chunks XOR-swizzled by (row mod 8), 8-row groups 1024 bytes apart.
//   Q tile (mt, kt): rows mt*128.., k = kt*64..   16 KB at ((mt*KT + kt) << 14)
//   S tile kt:       replicas 0..R-1, k = kt*64..  R*128 bytes at kt*R*128
#include <cuda_bf16.h>

#include <algorithm>
#include <numeric>
#include <queue>
#include <vector>

#include "vq_internal.cuh"

namespace vq {

namespace {

constexpr long long kWaitCycles = 4000000000LL;
enum { BT_ERR_PRODUCER = 1, BT_ERR_MMA = 2, BT_ERR_EPILOGUE = 4 };
constexpr int TILE_M = 128, TILE_KB = 128, TILE_K = 64;   // rows, bytes and bf16 elements of K per tile
constexpr uint32_t A_TILE = TILE_M * TILE_KB;             // 16 KB

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(uint64_t* b, uint32_t c) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(c) : "memory");
}
__device__ __forceinline__ void mb_expect(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mb_try(uint64_t* b, uint32_t par) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(par)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mb_wait(uint64_t* b, uint32_t par, int* err, int code) {
    const long long t0 = clock64();
    uint32_t spins = 0;
    while (!mb_try(b, par)) {
        if ((++spins & 1023u) == 0) {
            if (*(volatile int*)err) return false;
            if (clock64() - t0 > kWaitCycles) {
                atomicOr(err, code);
                return false;
            }
        }
    }
    return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(su32(dst)), "l"((uint64_t)src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}
// The same copy marked evict-first in L2: the coupling tiles stream through
// once per step, and should not push out the replica operand, which every row
// tile of the instance reads again.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void bulk_g2s_stream(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                                uint64_t pol) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
                 ::"r"(su32(dst)), "l"((uint64_t)src), "r"(bytes), "r"(su32(bar)), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void tcf_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tcf_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ uint64_t sdesc(const void* p) {
    const uint32_t a = su32(p);
    return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
           ((uint64_t)2 << 61);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void tld16(uint32_t t, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(t));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// byte offset of operand element (row r, k) inside a swizzled tile
__host__ __device__ __forceinline__ uint32_t swz(uint32_t r, uint32_t k) {
    return r * 128u + ((((k >> 3) ^ (r & 7u)) & 7u) << 4) + (k & 7u) * 2u;
}

struct BatchInst {
    int32_t n, MT, KT, pad;
    const uint8_t* qt;      // pre-tiled BF16 Qoff
    const float* bf;        // [n]
    float* S;               // [R][n]
    float* Y;               // [R][n]
    uint8_t* sop0;          // pre-tiled BF16 S operand, ping
    uint8_t* sop1;          // pong
    float c0;
    float pad2;
};

struct BatchArgs {
    const BatchInst* inst;
    const int32_t* order;       // instance ids, grouped by CTA
    const int32_t* cta_begin;   // [gridDim.x + 1]
    int32_t R, K;
    float dt, a0, sigma0;
    uint64_t seed;
    const float* a_table;
    int* err;
    float alpha;                // PA momentum
};

// METHOD: the integrator (veloxq_method), a template parameter so that the
// ballistic form keeps its own register allocation.
template <int STAGES, int METHOD>
__global__ void __launch_bounds__(192, 1) k_batch(const BatchArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int R = a.R;
    const uint32_t B_TILE = (uint32_t)R * TILE_KB;
    const uint32_t STAGE = A_TILE + B_TILE;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* accf = empty + STAGES;     // [2]
    uint64_t* acce = accf + 2;           // [2]
    uint64_t* stepr = acce + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(stepr + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int first = a.cta_begin[blockIdx.x], last = a.cta_begin[blockIdx.x + 1];
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(2 * R)) ncols <<= 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mb_init(&full[s], 1);
            mb_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mb_init(&accf[b], 1);
            mb_init(&acce[b], 4);
        }
        mb_init(stepr, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tcf_before();
    __syncthreads();
    tcf_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            const uint64_t qpol = l2_evict_first_policy();
            uint32_t it = 0, sp = 0;
            bool ok = true;
            for (int w = first; w < last && ok; ++w) {
                const BatchInst in = a.inst[a.order[w]];
                for (int k = 0; k < a.K && ok; ++k) {
                    if (!mb_wait(stepr, sp & 1u, a.err, BT_ERR_PRODUCER)) { ok = false; break; }
                    ++sp;
                    const uint8_t* sop = (k & 1) ? in.sop1 : in.sop0;
                    for (int mt = 0; mt < in.MT && ok; ++mt)
                        for (int kt = 0; kt < in.KT; ++kt) {
                            const uint32_t s = it % STAGES;
                            if (it >= (uint32_t)STAGES &&
                                !mb_wait(&empty[s], ((it / STAGES) - 1) & 1u, a.err, BT_ERR_PRODUCER)) {
                                ok = false;
                                break;
                            }
                            uint8_t* dst = smem + s * STAGE;
                            mb_expect(&full[s], STAGE);
                            bulk_g2s_stream(dst, in.qt + (((size_t)mt * in.KT + kt) << 14), A_TILE, &full[s], qpol);
                            bulk_g2s(dst + A_TILE, sop + (size_t)kt * B_TILE, B_TILE, &full[s]);
                            ++it;
                        }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(R >> 3) << 17) |
                                   ((uint32_t)(TILE_M >> 4) << 24);
            uint32_t it = 0, tt = 0;
            bool ok = true;
            for (int w = first; w < last && ok; ++w) {
                const BatchInst in = a.inst[a.order[w]];
                for (int k = 0; k < a.K && ok; ++k)
                    for (int mt = 0; mt < in.MT && ok; ++mt) {
                        const uint32_t b = tt & 1u;
                        if (tt >= 2 && !mb_wait(&acce[b], ((tt >> 1) - 1) & 1u, a.err, BT_ERR_MMA)) { ok = false; break; }
                        tcf_after();
                        const uint32_t d = tmem + b * (uint32_t)R;
                        for (int kt = 0; kt < in.KT; ++kt) {
                            const uint32_t s = it % STAGES;
                            if (!mb_wait(&full[s], (it / STAGES) & 1u, a.err, BT_ERR_MMA)) { ok = false; break; }
                            tcf_after();
                            const uint8_t* st = smem + s * STAGE;
#pragma unroll
                            for (int kk = 0; kk < TILE_KB / 32; ++kk)
                                mma_bf16(d, sdesc(st + kk * 32), sdesc(st + A_TILE + kk * 32), idesc,
                                         (kt | kk) != 0 ? 1u : 0u);
                            mma_commit(&empty[s]);
                            ++it;
                        }
                        if (!ok) break;
                        mma_commit(&accf[b]);
                        ++tt;
                    }
            }
        }
    } else {
        // epilogue: 4 warps, warp w owns tensor-memory lanes 32 (w % 4) .. +31
        const int q = warp & 3;
        const int et = threadIdx.x - 64;           // 0..127 among the epilogue warps
        uint32_t tt = 0;
        bool ok = true;
        for (int w = first; w < last && ok; ++w) {
            const BatchInst in = a.inst[a.order[w]];
            const int n = in.n;
            // initial state (Philox, as every other path) and the first operand
            for (int64_t e = et; e < (int64_t)R * n; e += 128) {
                const int r = (int)(e / n), i = (int)(e - (int64_t)r * n);
                float s0, y0;
                vqd::init_pair(i, r, a.seed, a.sigma0, &s0, &y0);
                in.S[e] = s0;
                in.Y[e] = y0;
                *reinterpret_cast<__nv_bfloat16*>(in.sop0 + (size_t)(i >> 6) * R * TILE_KB + swz(r, i & 63)) =
                    __float2bfloat16_rn(METHOD == vqd::METHOD_PA ? vqd::pa_sign(s0) : s0);
            }
            asm volatile("fence.proxy.async.global;" ::: "memory");
            epi_bar();
            if (et == 0) mb_arrive(stepr);
            for (int k = 0; k < a.K && ok; ++k) {
                const float a_k = __ldg(a.a_table + k);
                const float lam = METHOD == vqd::METHOD_PA ? vqd::pa_lambda(a_k, a.a0) : 0.0f;
                uint8_t* sop_n = (k & 1) ? in.sop0 : in.sop1;
                for (int mt = 0; mt < in.MT; ++mt) {
                    const uint32_t b = tt & 1u;
                    if (!mb_wait(&accf[b], (tt >> 1) & 1u, a.err, BT_ERR_EPILOGUE)) { ok = false; break; }
                    tcf_after();
                    const int row = mt * TILE_M + q * 32 + lane;
                    const bool row_ok = row < n;
                    const float bi = row_ok ? __ldg(in.bf + row) : 0.0f;
                    for (int c = 0; c < R / 16; ++c) {
                        uint32_t v[16];
                        tld16(tmem + ((uint32_t)(q * 32) << 16) + b * (uint32_t)R + (uint32_t)(c * 16), v);
                        float sv[16], yv[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int64_t p = (int64_t)(c * 16 + j) * n + row;
                            sv[j] = row_ok ? in.S[p] : 0.0f;
                            yv[j] = row_ok ? in.Y[p] : 0.0f;
                        }
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            float s = sv[j], y = yv[j];
                            const float F = __uint_as_float(v[j]);
                            if constexpr (METHOD == vqd::METHOD_PA) vqd::pa_update(F, bi, lam, a.dt, a.alpha, in.c0, s, y);
                            else if constexpr (METHOD == vqd::METHOD_ASB) vqd::asb_update(F, bi, a_k, a.dt, a.a0, in.c0, s, y);
                            else vqd::bsb_update(F, bi, a_k, a.dt, a.a0, in.c0, s, y);
                            if (row_ok) {
                                const int r = c * 16 + j;
                                const int64_t p = (int64_t)r * n + row;
                                in.S[p] = s;
                                in.Y[p] = y;
                                *reinterpret_cast<__nv_bfloat16*>(sop_n + (size_t)(row >> 6) * R * TILE_KB +
                                                                  swz(r, row & 63)) =
                                    __float2bfloat16_rn(METHOD == vqd::METHOD_PA ? vqd::pa_sign(s) : s);
                            }
                        }
                    }
                    tcf_before();
                    __syncwarp();
                    if (lane == 0) mb_arrive(&acce[b]);
                    ++tt;
                }
                if (!ok) break;
                if (k + 1 < a.K) {
                    // the next step's operand must be complete and visible to the bulk copies
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                    epi_bar();
                    if (et == 0) mb_arrive(stepr);
                }
            }
        }
    }
    tcf_before();
    __syncthreads();
    tcf_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// Qoff (FP32, [n][n]) -> pre-tiled BF16 operand; padding rows/columns are 0.
__global__ void k_tile_q(const float* __restrict__ q, int n, int MT, int KT, uint8_t* out) {
    const int tile = blockIdx.x;           // mt * KT + kt
    const int mt = tile / KT, kt = tile % KT;
    for (int e = threadIdx.x; e < TILE_M * TILE_K; e += blockDim.x) {
        const int r = e / TILE_K, k = e % TILE_K;
        const int gi = mt * TILE_M + r, gj = kt * TILE_K + k;
        const float v = (gi < n && gj < n) ? q[(size_t)gi * n + gj] : 0.0f;
        *reinterpret_cast<__nv_bfloat16*>(out + ((size_t)tile << 14) + swz(r, k)) = __float2bfloat16_rn(v);
    }
}

// stages + alignment slack + barriers (2 ST + 5 mbarriers and the tensor-memory slot)
template <int ST> size_t batch_smem(int R) {
    return (size_t)ST * (A_TILE + (size_t)R * TILE_KB) + 1024 + (size_t)(2 * ST + 5) * 8 + 16;
}

}  // namespace

bool batch_supported(veloxq_ctx* const* ctxs, int32_t count, int32_t R, const RunParams& p) {
    if (R < 16 || R > 128 || R % 16 != 0) return false;
    if (p.readout_every != 0 || p.prec != VELOXQ_PREC_BF16) return false;
    for (int m = 0; m < count; ++m)
        if (!ctxs[m] || !ctxs[m]->dense || ctxs[m]->n < 2 || ctxs[m]->n > 32768) return false;
    return true;
}

// Runs the persistent batched kernel, then the exact final-readout energies and
// the argmin of every instance. stages: 4 (two CTAs per SM) or 6 (one).
int batch_run(veloxq_ctx* const* ctxs, int32_t count, int32_t R, const RunParams& p, uint64_t seed, cudaStream_t st,
              int stages, DevBuf& work, int64_t* d_best_all, int* d_err, float* ms_main) {
    std::vector<BatchInst> host((size_t)count);
    std::vector<double> cost((size_t)count);
    for (int m = 0; m < count; ++m) {
        veloxq_ctx* c = ctxs[m];
        const int n = (int)c->n;
        const int MT = (int)div_up(n, TILE_M), KT = (int)div_up(n, TILE_K);
        const size_t qbytes = (size_t)MT * KT * A_TILE;
        if (c->qtile_bytes != qbytes) {
            VQ_TRY(c->qtile.ensure(qbytes));
            k_tile_q<<<(unsigned)(MT * KT), 256, 0, st>>>(c->qoff32.as<float>(), n, MT, KT, c->qtile.as<uint8_t>());
            VQ_LAUNCH_CHECK("tile Q");
            c->qtile_bytes = qbytes;
        }
        const size_t sopb = (size_t)KT * R * TILE_KB;
        VQ_TRY(c->s_a.ensure(sizeof(float) * (size_t)R * n));
        VQ_TRY(c->y.ensure(sizeof(float) * (size_t)R * n));
        VQ_TRY(c->sop_a.ensure(sopb));
        VQ_TRY(c->sop_b.ensure(sopb));
        VQ_CUDA(cudaMemsetAsync(c->sop_a.p, 0, sopb, st));   // K padding stays 0
        VQ_CUDA(cudaMemsetAsync(c->sop_b.p, 0, sopb, st));
        BatchInst b{};
        b.n = n;
        b.MT = MT;
        b.KT = KT;
        b.qt = c->qtile.as<uint8_t>();
        b.bf = c->bf.as<float>();
        b.S = c->s_a.as<float>();
        b.Y = c->y.as<float>();
        b.sop0 = c->sop_a.as<uint8_t>();
        b.sop1 = c->sop_b.as<uint8_t>();
        b.c0 = p.c0 > 0 && p.c0_given ? p.c0 : (c->rho > 1e-12 ? (float)(2.0 * p.kappa / c->rho) : p.kappa);
        host[m] = b;
        cost[m] = (double)MT * KT + 4.0;   // tiles per step plus a fixed per-step latency
        c->batch_R = R;
    }
    // longest processing time first onto the least loaded CTA
    const int ctas = device_sms(ctxs[0]->device) * (stages == 4 ? 2 : 1);
    std::vector<int> idx((size_t)count);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    using Item = std::pair<double, int>;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
    for (int c = 0; c < ctas; ++c) heap.push({0.0, c});
    std::vector<std::vector<int>> lists((size_t)ctas);
    for (int m : idx) {
        Item t = heap.top();
        heap.pop();
        lists[t.second].push_back(m);
        heap.push({t.first + cost[m], t.second});
    }
    std::vector<int32_t> order, begin(1, 0);
    for (auto& l : lists) {
        for (int m : l) order.push_back(m);
        begin.push_back((int32_t)order.size());
    }
    const size_t ib = sizeof(BatchInst) * (size_t)count, ob = sizeof(int32_t) * order.size(),
                 bb = sizeof(int32_t) * begin.size();
    VQ_TRY(work.ensure(ib + ob + bb + 64));
    uint8_t* w = work.as<uint8_t>();
    VQ_CUDA(cudaMemcpyAsync(w, host.data(), ib, cudaMemcpyHostToDevice, st));
    VQ_CUDA(cudaMemcpyAsync(w + ib, order.data(), ob, cudaMemcpyHostToDevice, st));
    VQ_CUDA(cudaMemcpyAsync(w + ib + ob, begin.data(), bb, cudaMemcpyHostToDevice, st));
    BatchArgs a;
    a.inst = reinterpret_cast<const BatchInst*>(w);
    a.order = reinterpret_cast<const int32_t*>(w + ib);
    a.cta_begin = reinterpret_cast<const int32_t*>(w + ib + ob);
    a.R = R;
    a.K = p.K;
    a.dt = p.dt;
    a.a0 = p.a0;
    a.sigma0 = p.sigma0;
    a.seed = seed;
    a.a_table = ctxs[0]->a_table.as<float>();
    a.err = d_err;
    a.alpha = p.alpha;
    cudaEvent_t e0, e1;
    VQ_CUDA(cudaEventCreate(&e0));
    VQ_CUDA(cudaEventCreate(&e1));
    VQ_CUDA(cudaEventRecord(e0, st));
    void (*fn)(const BatchArgs);
    const int m = p.method;
    if (stages == 4) fn = m == VELOXQ_METHOD_PA ? k_batch<4, vqd::METHOD_PA> : m == VELOXQ_METHOD_ASB ? k_batch<4, vqd::METHOD_ASB> : k_batch<4, vqd::METHOD_BSB>;
    else fn = m == VELOXQ_METHOD_PA ? k_batch<6, vqd::METHOD_PA> : m == VELOXQ_METHOD_ASB ? k_batch<6, vqd::METHOD_ASB> : k_batch<6, vqd::METHOD_BSB>;
    const size_t smem = stages == 4 ? batch_smem<4>(R) : batch_smem<6>(R);
    VQ_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    fn<<<ctas, 192, smem, st>>>(a);
    VQ_LAUNCH_CHECK("batch kernel");
    VQ_CUDA(cudaEventRecord(e1, st));
    // exact final-readout energies and the best replica of every instance
    for (int m = 0; m < count; ++m) {
        veloxq_ctx* c = ctxs[m];
        const int np = (int)div_up(c->n, 64);
        VQ_TRY(c->ework.ensure(sizeof(int64_t) * (size_t)np * R));
        VQ_TRY(c->best_e.ensure(sizeof(int64_t) * R));
        VQ_TRY(c->flags.ensure((size_t)R));
        VQ_TRY(c->best_bits.ensure(sizeof(uint32_t) * (size_t)R * div_up(c->n, 32)));
        VQ_TRY(c->misc.ensure(sizeof(int64_t) * 16));
        VQ_TRY(c->xout.ensure((size_t)c->n));
        cudaStream_t keep = c->stream;
        c->stream = st;
        int np2 = 0;
        int rc = dense_energy(c, R, c->s_a.as<float>(), c->ework.as<int64_t>(), &np2, false);
        if (rc == VELOXQ_OK) rc = (cudaMemsetAsync(c->best_e.p, 0x7f, sizeof(int64_t) * R, st) == cudaSuccess)
                                      ? VELOXQ_OK : VELOXQ_ECUDA;
        if (rc == VELOXQ_OK) rc = launch_best_update(c, R, np2, c->ework.as<int64_t>(), c->best_e.as<int64_t>(),
                                                     c->flags.as<uint8_t>());
        if (rc == VELOXQ_OK) rc = launch_best_bits(c, R, LAYOUT_RN, c->s_a.as<float>(), c->flags.as<uint8_t>(),
                                                   c->best_bits.as<uint32_t>());
        if (rc == VELOXQ_OK) rc = launch_argmin_unpack(c, R, c->best_e.as<int64_t>(), c->best_bits.as<uint32_t>(),
                                                       c->misc.as<int64_t>(), c->xout.as<uint8_t>());
        c->stream = keep;
        if (rc != VELOXQ_OK) return rc;
        VQ_CUDA(cudaMemcpyAsync(d_best_all + 2 * m, c->misc.p, 2 * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    }
    VQ_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    VQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms_main) *ms_main = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return VELOXQ_OK;
}

}  // namespace vq
