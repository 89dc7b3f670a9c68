// vq_batch.cu -- many dense instances of uneven size in ONE persistent launch
// (BF16 or FP8 E4M3 tensor-core field, FP32 state, fused update).
//
// Each CTA owns a list of whole instances (no synchronisation between CTAs);
// the host assigns instances to CTAs longest-first (LPT on n^2). For each
// instance and step, the CTA walks its 128-row tiles: warp 0 streams the
// pre-tiled operands with 1-D bulk copies, warp 1 issues the MMAs
// (M = 128 variables, N = R replicas, K = variables) into one of two tensor
// memory buffers, warps 2-5 (2-9 in the 6-stage form) read the other buffer
// back and update their rows
// (the epilogue of tile t overlaps the main loop of tile t + 1). After the
// last tile of a step the epilogue warps publish the next operand (a proxy
// fence and a named barrier) before the producer may read it.
//
// Operand layout in global memory (the layout the MMA reads from shared
// memory, so that a plain bulk copy lands it there): 128-byte rows, 16-byte
// chunks XOR-swizzled by (row mod 8), 8-row groups 1024 bytes apart. A row
// holds TK = 64 BF16 or 128 E4M3 elements of K.
//   Q tile (mt, kt): rows mt*128.., k = kt*TK..   16 KB at ((mt*KT + kt) << 14)
//   S tile kt:       replicas 0..R-1, k = kt*TK..  R*128 bytes at kt*R*128
//   (two FP8 terms of S: the lo plane follows the hi plane, KT*R*128 bytes on)
// FP8: Qoff_ij / q_i in E4M3 with q_i = amax_i / 448, S as v = 448 s in one
// E4M3 term or two (hi = e4m3(v), lo = e4m3(v - hi), both multiplied by the
// same Q tile into the same accumulator), F_i = acc q_i / 448: the same
// arithmetic as the single-instance tensor-core step.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <queue>
#include <vector>

#include "vq_async.cuh"
#include "vq_internal.cuh"

namespace vq {

namespace {

enum { BT_ERR_PRODUCER = 1, BT_ERR_MMA = 2, BT_ERR_EPILOGUE = 4 };
constexpr int TILE_M = 128, TILE_KB = 128;                // rows and bytes of K per tile
constexpr uint32_t A_TILE = TILE_M * TILE_KB;             // 16 KB
template <int PREC> constexpr int tile_k() { return PREC == 1 ? 64 : 128; }   // elements of K per tile

using vqa::bulk_g2s;
using vqa::bulk_g2s_stream;
using vqa::l2_evict_first_policy;
using vqa::mb_arrive;
using vqa::mb_expect;
using vqa::mb_init;
using vqa::mb_try;
using vqa::mb_wait;
using vqa::su32;
// (bulk_g2s_stream with an evict-first policy: the coupling tiles stream
// through once per step, and should not push out the replica operand, which
// every row tile of the instance reads again)
__device__ __forceinline__ void tcf_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tcf_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ uint64_t sdesc(const void* p) {
    const uint32_t a = su32(p);
    return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
           ((uint64_t)2 << 61);
}
template <int PREC>
__device__ __forceinline__ void mma_tile(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (PREC == 1) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
            ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n"
            ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void tld8(uint32_t t, uint32_t (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(t));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
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
// Epilogue warps: 8 in the 6-stage form (one CTA per SM; two warps per
// quarter of the tensor-memory lanes, each taking half of the replica
// chunks), 4 in the 4-stage form (two CTAs per SM share the registers).
template <int STAGES> constexpr int epi_warps() { return STAGES == 6 ? 8 : 4; }
template <int STAGES> constexpr int batch_threads() { return 64 + 32 * epi_warps<STAGES>(); }
template <int STAGES> __device__ __forceinline__ void epi_bar() {
    asm volatile("bar.sync 1, %0;" ::"n"(32 * epi_warps<STAGES>()) : "memory");
}

// byte offset of operand element (row r, k) inside a swizzled tile, for
// elements of EB bytes
template <int EB> __host__ __device__ __forceinline__ uint32_t swz(uint32_t r, uint32_t k) {
    const uint32_t b = k * (uint32_t)EB;
    return r * 128u + ((((b >> 4) ^ (r & 7u)) & 7u) << 4) + (b & 15u);
}

// The next operand of one state value: bf16(s); or v = 448 s as hi =
// e4m3(v) and, with two terms, lo = e4m3(v - hi) `plane` bytes further.
template <int PREC, int TERMS>
__device__ __forceinline__ void put_op(uint8_t* at, size_t plane, float s) {
    if constexpr (PREC == 1) {
        *reinterpret_cast<__nv_bfloat16*>(at) = __float2bfloat16_rn(s);
    } else {
        const float v = __fmul_rn(448.0f, s);
        const __nv_fp8_storage_t hi = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
        at[0] = hi;
        if constexpr (TERMS == 2) {
            const float hf = __half2float(__half(__nv_cvt_fp8_to_halfraw(hi, __NV_E4M3)));
            at[plane] = __nv_cvt_float_to_fp8(__fsub_rn(v, hf), __NV_SATFINITE, __NV_E4M3);
        }
    }
}

struct BatchInst {
    int32_t n, MT, KT, pad;
    const uint8_t* qt;      // pre-tiled Qoff operand (BF16, or E4M3 of Qoff_ij / q_i)
    const float* qs;        // [n] FP8 row scales q_i = amax_i / 448 (FP8 only)
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
    const int32_t* order;       // work items (instance id * G + replica group), grouped by CTA
    const int32_t* cta_begin;   // [gridDim.x + 1]
    int32_t R, K;               // replicas of every instance, steps
    int32_t G, RG;              // replica groups per instance and replicas per group (R = G RG)
    float dt, a0, sigma0;
    const uint64_t* seed;       // device: the Philox key of this solve (uploaded per solve, so that a
                                // captured graph of the launch serves every seed)
    const float* a_table;
    int* err;
    float alpha;                // PA momentum
};

// METHOD: the integrator (veloxq_method), a template parameter so that the
// ballistic form keeps its own register allocation. PREC: 1 BF16, 2 E4M3;
// TERMS: E4M3 terms of S (1 or 2).
template <int PREC, int TERMS, int STAGES, int METHOD>
__global__ void __launch_bounds__(batch_threads<STAGES>(), STAGES == 4 ? 2 : 1) k_batch(const BatchArgs a) {
    constexpr int EB = PREC == 1 ? 2 : 1;
    constexpr int TK = tile_k<PREC>();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    // A work item is one replica group of one instance: RG replicas, the
    // MMA's N. Replicas are independent, so the groups of an instance need no
    // coordination: each reads the instance's couplings and its own rows of
    // the operand tiles (RG rows at r0 inside every R-row tile), and writes
    // only its replicas' state.
    const int R = a.RG;
    const uint32_t B_TILE = (uint32_t)R * TILE_KB;               // one group's rows of an operand tile
    const uint32_t B_STRIDE = (uint32_t)a.R * TILE_KB;           // one operand tile (all replicas)
    const uint32_t STAGE = A_TILE + TERMS * B_TILE;
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
            mb_init(&acce[b], epi_warps<STAGES>());
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
                const int item = a.order[w];
                const BatchInst in = a.inst[item / a.G];
                const size_t r0b = (size_t)(item % a.G) * B_TILE;      // this group's rows in a tile
                const size_t lo_off = (size_t)in.KT * B_STRIDE;       // lo plane of a two-term operand
                for (int k = 0; k < a.K && ok; ++k) {
                    if (!mb_wait(stepr, sp & 1u, a.err, BT_ERR_PRODUCER)) { ok = false; break; }
                    ++sp;
                    const uint8_t* sop = ((k & 1) ? in.sop1 : in.sop0) + r0b;
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
                            bulk_g2s(dst + A_TILE, sop + (size_t)kt * B_STRIDE, B_TILE, &full[s]);
                            if constexpr (TERMS == 2)
                                bulk_g2s(dst + A_TILE + B_TILE, sop + lo_off + (size_t)kt * B_STRIDE, B_TILE,
                                         &full[s]);
                            ++it;
                        }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // D F32; A, B BF16 (kind::f16) or E4M3 (kind::f8f6f4, format 0); K-major; N = R; M = 128
            const uint32_t idesc = (1u << 4) | ((PREC == 1 ? 1u : 0u) << 7) | ((PREC == 1 ? 1u : 0u) << 10) |
                                   ((uint32_t)(R >> 3) << 17) | ((uint32_t)(TILE_M >> 4) << 24);
            uint32_t it = 0, tt = 0;
            bool ok = true;
            for (int w = first; w < last && ok; ++w) {
                const BatchInst in = a.inst[a.order[w] / a.G];
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
                            for (int kk = 0; kk < TILE_KB / 32; ++kk) {
                                const uint64_t da = sdesc(st + kk * 32);
                                mma_tile<PREC>(d, da, sdesc(st + A_TILE + kk * 32), idesc, (kt | kk) != 0 ? 1u : 0u);
                                if constexpr (TERMS == 2)
                                    mma_tile<PREC>(d, da, sdesc(st + A_TILE + B_TILE + kk * 32), idesc, 1u);
                            }
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
        constexpr int EW = epi_warps<STAGES>();
        const int q = warp & 3;                    // tensor-memory lanes 32 q .. 32 q + 31
        const int half = (warp - 2) >> 2;          // with 8 warps: which half of the replica chunks
        const int et = threadIdx.x - 64;           // 0 .. 32 EW - 1 among the epilogue warps
        uint32_t tt = 0;
        bool ok = true;
        for (int w = first; w < last && ok; ++w) {
            const int item = a.order[w];
            const BatchInst in = a.inst[item / a.G];
            const int n = in.n;
            const int r0 = (item % a.G) * R;                       // first replica of the group
            const size_t lo_off = (size_t)in.KT * B_STRIDE;
            float* const S = in.S + (int64_t)r0 * n;              // the group's rows of [R][n]
            float* const Y = in.Y + (int64_t)r0 * n;
            // initial state (Philox with the instance's replica index, as every
            // other path) and the first operand
            for (int64_t e = et; e < (int64_t)R * n; e += 32 * EW) {
                const int r = (int)(e / n), i = (int)(e - (int64_t)r * n);
                float s0, y0;
                vqd::init_pair(i, r0 + r, *a.seed, a.sigma0, &s0, &y0);
                S[e] = s0;
                Y[e] = y0;
                put_op<PREC, TERMS>(in.sop0 + (size_t)(i / TK) * B_STRIDE + swz<EB>(r0 + r, i % TK), lo_off,
                                    METHOD == vqd::METHOD_PA ? vqd::pa_sign(s0) : s0);
            }
            asm volatile("fence.proxy.async.global;" ::: "memory");
            epi_bar<STAGES>();
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
                    // F = acc q_i / 448 (Qoff scaled by q_i, S by 448)
                    const float fscale = (PREC == 2 && row_ok) ? __ldg(in.qs + row) * (1.0f / 448.0f) : 1.0f;
                    uint8_t* op_row = sop_n + (size_t)(row / TK) * B_STRIDE;
                    // the state of CW replicas at a time: with 8 epilogue warps
                    // (each half of the chunks) 8 at a time, the next chunk's
                    // loads issued before this one is updated; with 4 warps 16
                    constexpr int CW = EW == 8 ? 8 : 16;
                    constexpr bool AHEAD = EW == 8;
                    const int nch = R / CW;
                    const int c_lo = EW == 8 ? half * ((nch + 1) / 2) : 0;
                    const int c_hi = EW == 8 ? min(nch, c_lo + (nch + 1) / 2) : nch;
                    float sv[CW], yv[CW];
                    auto load_chunk = [&](int c, float (&sd)[CW], float (&yd)[CW]) {
#pragma unroll
                        for (int j = 0; j < CW; ++j) {
                            const int64_t p = (int64_t)(c * CW + j) * n + row;
                            sd[j] = row_ok ? S[p] : 0.0f;
                            yd[j] = row_ok ? Y[p] : 0.0f;
                        }
                    };
                    if constexpr (AHEAD) {
                        if (c_lo < c_hi) load_chunk(c_lo, sv, yv);
                    }
                    for (int c = c_lo; c < c_hi; ++c) {
                        uint32_t v[CW];
                        const uint32_t tcol = tmem + ((uint32_t)(q * 32) << 16) + b * (uint32_t)R + (uint32_t)(c * CW);
                        if constexpr (CW == 8) tld8(tcol, v);
                        else tld16(tcol, v);
                        float sn[CW], yn[CW];
                        if constexpr (AHEAD) {
                            if (c + 1 < c_hi) load_chunk(c + 1, sn, yn);
                        } else {
                            load_chunk(c, sv, yv);
                        }
#pragma unroll
                        for (int j = 0; j < CW; ++j) {
                            float s = sv[j], y = yv[j];
                            const float F = __uint_as_float(v[j]) * fscale;
                            if constexpr (METHOD == vqd::METHOD_PA) vqd::pa_update(F, bi, lam, a.dt, a.alpha, in.c0, s, y);
                            else if constexpr (METHOD == vqd::METHOD_ASB) vqd::asb_update(F, bi, a_k, a.dt, a.a0, in.c0, s, y);
                            else vqd::bsb_update(F, bi, a_k, a.dt, a.a0, in.c0, s, y);
                            if (row_ok) {
                                const int r = c * CW + j;
                                const int64_t p = (int64_t)r * n + row;
                                S[p] = s;
                                Y[p] = y;
                                put_op<PREC, TERMS>(op_row + swz<EB>(r0 + r, row % TK), lo_off,
                                                    METHOD == vqd::METHOD_PA ? vqd::pa_sign(s) : s);
                            }
                        }
                        if constexpr (AHEAD) {
#pragma unroll
                            for (int j = 0; j < CW; ++j) {
                                sv[j] = sn[j];
                                yv[j] = yn[j];
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
                    epi_bar<STAGES>();
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
    constexpr int TK = tile_k<1>();
    const int tile = blockIdx.x;           // mt * KT + kt
    const int mt = tile / KT, kt = tile % KT;
    for (int e = threadIdx.x; e < TILE_M * TK; e += blockDim.x) {
        const int r = e / TK, k = e % TK;
        const int gi = mt * TILE_M + r, gj = kt * TK + k;
        const float v = (gi < n && gj < n) ? q[(size_t)gi * n + gj] : 0.0f;
        *reinterpret_cast<__nv_bfloat16*>(out + ((size_t)tile << 14) + swz<2>(r, k)) = __float2bfloat16_rn(v);
    }
}

// Per-row FP8 scale q_i = amax_i / 448 (1 for an all-zero row), the same
// values as the single-instance FP8 operand.
__global__ void k_row_scale(const float* __restrict__ q, int n, float* scale) {
    __shared__ float sh[256];
    const int64_t i = blockIdx.x;
    float m = 0.0f;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) m = fmaxf(m, fabsf(q[i * n + j]));
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) scale[i] = sh[0] > 0.0f ? sh[0] / 448.0f : 1.0f;
}

// Qoff -> pre-tiled E4M3 operand e4m3(Qoff_ij / q_i); padding is 0.
__global__ void k_tile_q8(const float* __restrict__ q, int n, int MT, int KT, const float* __restrict__ scale,
                          uint8_t* out) {
    constexpr int TK = tile_k<2>();
    const int tile = blockIdx.x;
    const int mt = tile / KT, kt = tile % KT;
    for (int e = threadIdx.x; e < TILE_M * TK; e += blockDim.x) {
        const int r = e / TK, k = e % TK;
        const int gi = mt * TILE_M + r, gj = kt * TK + k;
        float v = 0.0f;
        if (gi < n && gj < n) v = q[(size_t)gi * n + gj] * (1.0f / scale[gi]);
        out[((size_t)tile << 14) + swz<1>(r, k)] = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    }
}

// stages + alignment slack + barriers (2 ST + 5 mbarriers and the tensor-memory slot)
size_t batch_smem(int stages, int terms, int R) {
    return (size_t)stages * (A_TILE + (size_t)terms * R * TILE_KB) + 1024 + (size_t)(2 * stages + 5) * 8 + 16;
}
constexpr size_t kBatchSmemMax = 227 * 1024;

using BatchKernel = void (*)(const BatchArgs);
template <int PREC, int TERMS, int ST> BatchKernel pick_batch(int m) {
    if constexpr (PREC == 2) {
        // E4M3 with two S terms runs the ballistic form; PA's exact operand needs one term
        if (m == VELOXQ_METHOD_PA) return k_batch<PREC, TERMS, ST, vqd::METHOD_PA>;
        return k_batch<PREC, TERMS, ST, vqd::METHOD_BSB>;
    } else {
        if (m == VELOXQ_METHOD_PA) return k_batch<PREC, TERMS, ST, vqd::METHOD_PA>;
        if (m == VELOXQ_METHOD_ASB) return k_batch<PREC, TERMS, ST, vqd::METHOD_ASB>;
        return k_batch<PREC, TERMS, ST, vqd::METHOD_BSB>;
    }
}
// The kernel of a batch form: operand precision, S terms, pipeline stages, integrator.
BatchKernel batch_kernel(int prec, int terms, int stages, int method) {
    if (prec == VELOXQ_PREC_BF16) return stages == 4 ? pick_batch<1, 1, 4>(method) : pick_batch<1, 1, 6>(method);
    if (terms == 2) return stages == 4 ? pick_batch<2, 2, 4>(method) : pick_batch<2, 2, 6>(method);
    return stages == 4 ? pick_batch<2, 1, 4>(method) : pick_batch<2, 1, 6>(method);
}

// ---- the final readout of every instance in two launches ------------------
// Exact energies of x_r = [S_r > 0] in the same fixed point as a single
// context's readout: parts[g][r] = sum over the 64 rows of tile g of
// x_ri (dfix_i + sum_{j != i} round(Q_ij 2^shift) x_rj), Q as given. A block
// takes one (instance, 64-row tile, 32-replica tile) item of the work list.
struct ReadInst {
    const void* q;           // [n][n] Q as given (element type of the launch)
    const int64_t* dfix;     // [n]
    const float* S;          // [R][n] final state
    int64_t* parts;          // [ceil(n / 64)][R]
    uint8_t* x;              // [n] winner's vector
    int32_t n, shift;
};
template <typename QT>
__global__ void __launch_bounds__(256) k_batch_energy(const ReadInst* __restrict__ insts,
                                                      const int32_t* __restrict__ work, int32_t R) {
    __shared__ int64_t qt[64][33];
    __shared__ uint32_t xw[32];
    __shared__ int64_t red[8][32];
    const int32_t m = work[2 * blockIdx.x], local = work[2 * blockIdx.x + 1];
    const ReadInst in = insts[m];
    const int32_t n = in.n;
    const int32_t tiles = (n + 63) / 64;
    const int32_t tile = local % tiles, rt = local / tiles;
    const QT* Q = static_cast<const QT*>(in.q);
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int32_t r = rt * 32 + lane;
    const int64_t i0 = (int64_t)tile * 64;
    int64_t row[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) row[q] = 0;
    for (int64_t j0 = 0; j0 < n; j0 += 32) {
        __syncthreads();
        for (int e = threadIdx.x; e < 64 * 32; e += 256) {
            const int ii = e / 32, jj = e % 32;
            const int64_t gi = i0 + ii, gj = j0 + jj;
            qt[ii][jj] = (gi < n && gj < n && gi != gj) ? vqd::qfix<QT>(Q[gi * n + gj], in.shift) : 0;
        }
        if (g == 0) {
            uint32_t w = 0;
            if (r < R)
                for (int jj = 0; jj < 32; ++jj) {
                    const int64_t gj = j0 + jj;
                    if (gj < n && in.S[(int64_t)r * n + gj] > 0.0f) w |= 1u << jj;
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
            if (gi < n && in.S[(int64_t)r * n + gi] > 0.0f) part += __ldg(in.dfix + gi) + row[q];
        }
    }
    red[g][lane] = part;
    __syncthreads();
    if (g == 0 && r < R) {
        int64_t tot = 0;
        for (int q = 0; q < 8; ++q) tot += red[q][lane];
        in.parts[(int64_t)tile * R + r] = tot;
    }
}

// One block per instance: each replica's energy (its parts summed), the
// lowest energy with the lowest replica index on ties, that replica's
// readout x = [S > 0], and (replica, fixed-point energy) into best[2 m ..].
__global__ void __launch_bounds__(256) k_batch_finish(const ReadInst* __restrict__ insts, int32_t R,
                                                      int64_t* __restrict__ best) {
    __shared__ int64_t sv[256];
    __shared__ int32_t si[256];
    const int32_t m = blockIdx.x;
    const ReadInst in = insts[m];
    const int32_t tiles = (in.n + 63) / 64;
    int64_t bv = INT64_MAX;
    int32_t bi = INT32_MAX;
    for (int32_t r = threadIdx.x; r < R; r += blockDim.x) {
        int64_t tot = 0;
        for (int32_t t = 0; t < tiles; ++t) tot += in.parts[(int64_t)t * R + r];
        if (tot < bv || (tot == bv && r < bi)) {
            bv = tot;
            bi = r;
        }
    }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
        if (threadIdx.x < s2) {
            const int64_t v = sv[threadIdx.x + s2];
            const int32_t i = si[threadIdx.x + s2];
            if (v < sv[threadIdx.x] || (v == sv[threadIdx.x] && i < si[threadIdx.x])) {
                sv[threadIdx.x] = v;
                si[threadIdx.x] = i;
            }
        }
        __syncthreads();
    }
    const int32_t rb = si[0];
    for (int32_t i = threadIdx.x; i < in.n; i += blockDim.x)
        in.x[i] = in.S[(int64_t)rb * in.n + i] > 0.0f ? 1 : 0;
    if (threadIdx.x == 0) {
        best[2 * m] = rb;
        best[2 * m + 1] = sv[0];
    }
}

}  // namespace

int batch_terms(int prec, int method) {
    return prec == VELOXQ_PREC_FP8 && method != VELOXQ_METHOD_PA ? 2 : 1;
}

// Whether a batch form fits one CTA's shared memory.
bool batch_stages_fit(int prec, int method, int stages, int32_t R) {
    return batch_smem(stages, batch_terms(prec, method), R) <= kBatchSmemMax;
}

bool batch_supported(veloxq_ctx* const* ctxs, int32_t count, int32_t R, const RunParams& p) {
    if (R < 16 || R > 128 || R % 16 != 0) return false;
    if (p.readout_every != 0) return false;
    if (p.prec != VELOXQ_PREC_BF16 && p.prec != VELOXQ_PREC_FP8 && p.prec != VELOXQ_PREC_FP8_ONE_TERM) return false;
    if (p.prec != VELOXQ_PREC_BF16 && p.method == VELOXQ_METHOD_ASB) return false;
    if (!batch_stages_fit(p.prec, p.method, 4, R)) return false;
    for (int m = 0; m < count; ++m)
        if (!ctxs[m] || !ctxs[m]->dense || ctxs[m]->n < 2 || ctxs[m]->n > 32768) return false;
    return true;
}

// Runs the persistent batched kernel, then the exact final-readout energies and
// the argmin of every instance. stages: 4 (two CTAs per SM) or 6 (one).
int batch_run(veloxq_ctx* const* ctxs, int32_t count, int32_t R, const RunParams& p, uint64_t seed, cudaStream_t st,
              int stages, int split, DevBuf& work, int64_t* d_best_all, int* d_err, float* ms_main,
              int64_t* launches, BatchGraph* graph) {
    int64_t nl = 0;
    std::vector<std::pair<void*, size_t>> zero;   // operand buffers whose padding is zeroed
    const int terms = batch_terms(p.prec, p.method);
    if (split < 1 || R % split != 0 || (R / split) % 16 != 0)
        return fail(VELOXQ_EINVAL, "replica groups must hold a multiple of 16 replicas");
    const int RG = R / split;
    if (!batch_stages_fit(p.prec, p.method, stages, RG)) return fail(VELOXQ_EINVAL, "batch stages exceed shared memory");
    BatchKernel fn = batch_kernel(p.prec, terms, stages, p.method);
    const size_t smem = batch_smem(stages, terms, RG);
    VQ_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    VQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, stages == 6 ? batch_threads<6>() : batch_threads<4>(),
                                                          smem));
    if (per_sm < 1) return fail(VELOXQ_EUNSUPPORTED, "the batched kernel does not fit an SM");
    std::vector<BatchInst> host((size_t)count);
    std::vector<double> cost((size_t)count);
    for (int m = 0; m < count; ++m) {
        veloxq_ctx* c = ctxs[m];
        const int n = (int)c->n;
        const int fp8 = p.prec == VELOXQ_PREC_BF16 ? 0 : 1;
        const int MT = (int)div_up(n, TILE_M), KT = (int)div_up(n, fp8 ? tile_k<2>() : tile_k<1>());
        const size_t qbytes = (size_t)MT * KT * A_TILE;
        if (c->qtile_bytes != qbytes || c->qtile_fp8 != fp8) {
            VQ_TRY(c->qtile.ensure(qbytes));
            if (fp8) {
                VQ_TRY(c->qscale8.ensure(sizeof(float) * (size_t)n));
                k_row_scale<<<(unsigned)n, 256, 0, st>>>(c->qoff32.as<float>(), n, c->qscale8.as<float>());
                k_tile_q8<<<(unsigned)(MT * KT), 256, 0, st>>>(c->qoff32.as<float>(), n, MT, KT,
                                                               c->qscale8.as<float>(), c->qtile.as<uint8_t>());
            } else {
                k_tile_q<<<(unsigned)(MT * KT), 256, 0, st>>>(c->qoff32.as<float>(), n, MT, KT,
                                                              c->qtile.as<uint8_t>());
            }
            VQ_LAUNCH_CHECK("tile Q");
            nl += fp8 ? 2 : 1;
            c->qtile_bytes = qbytes;
            c->qtile_fp8 = fp8;
        }
        const size_t sopb = (size_t)terms * KT * R * TILE_KB;
        VQ_TRY(c->s_a.ensure(sizeof(float) * (size_t)R * n));
        VQ_TRY(c->y.ensure(sizeof(float) * (size_t)R * n));
        void* pa = c->sop_a.p;
        void* pb = c->sop_b.p;
        VQ_TRY(c->sop_a.ensure(sopb));
        VQ_TRY(c->sop_b.ensure(sopb));
        // the K padding of the operand tiles is never written: zero it when the
        // buffers last held another layout (or were just allocated); a captured
        // launch zeroes it on every replay
        const int64_t tag = ((int64_t)R << 16) | ((int64_t)p.prec << 8) | ((int64_t)terms << 4) | 1;
        if (graph || c->sop_tag != tag || c->sop_a.p != pa || c->sop_b.p != pb) {
            zero.push_back({c->sop_a.p, sopb});
            zero.push_back({c->sop_b.p, sopb});
            c->sop_tag = tag;
        }
        BatchInst b{};
        b.n = n;
        b.MT = MT;
        b.KT = KT;
        b.qt = c->qtile.as<uint8_t>();
        b.qs = fp8 ? c->qscale8.as<float>() : nullptr;
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
    // work items (instance, replica group), longest processing time first onto
    // the least loaded CTA; a group streams all of its instance's couplings,
    // so it costs as much as a whole instance
    const int ctas = device_sms(ctxs[0]->device) * per_sm;
    const int items = count * split;
    std::vector<int> idx((size_t)items);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return cost[x / split] > cost[y / split]; });
    using Item = std::pair<double, int>;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
    for (int c = 0; c < ctas; ++c) heap.push({0.0, c});
    std::vector<std::vector<int>> lists((size_t)ctas);
    for (int m : idx) {
        Item t = heap.top();
        heap.pop();
        lists[t.second].push_back(m);
        heap.push({t.first + cost[m / split], t.second});
    }
    std::vector<int32_t> order, begin(1, 0);
    for (auto& l : lists) {
        for (int m : l) order.push_back(m);
        begin.push_back((int32_t)order.size());
    }
    // the final readout's tables: one entry per instance, and per element type
    // of Q a work list of (instance, 64-row tile, 32-replica tile) items
    std::vector<ReadInst> rd((size_t)count);
    std::vector<int32_t> rwork[4];
    for (int m = 0; m < count; ++m) {
        veloxq_ctx* c = ctxs[m];
        const int tiles = (int)div_up(c->n, 64);
        VQ_TRY(c->ework.ensure(sizeof(int64_t) * (size_t)tiles * R));
        VQ_TRY(c->xout.ensure((size_t)c->n));
        rd[m] = ReadInst{c->qx.p, c->dfix.as<int64_t>(), c->s_a.as<float>(), c->ework.as<int64_t>(),
                         c->xout.as<uint8_t>(), (int32_t)c->n, c->energy_shift};
        const int t = (int)c->qx_type;
        if (t < 0 || t > 3) return fail(VELOXQ_EINVAL, "unknown coupling type");
        for (int l = 0; l < tiles * (int)div_up(R, 32); ++l) {
            rwork[t].push_back(m);
            rwork[t].push_back(l);
        }
    }
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t ib = al(sizeof(BatchInst) * (size_t)count), ob = al(sizeof(int32_t) * order.size()),
                 bb = al(sizeof(int32_t) * begin.size()), rb = al(sizeof(ReadInst) * (size_t)count);
    size_t wb[4], wtot = 0;
    for (int t = 0; t < 4; ++t) {
        wb[t] = al(sizeof(int32_t) * rwork[t].size());
        wtot += wb[t];
    }
    VQ_TRY(work.ensure(ib + ob + bb + rb + wtot + 64));
    uint8_t* w = work.as<uint8_t>();
    uint64_t* seed_dev = reinterpret_cast<uint64_t*>(w + ib + ob + bb + rb + wtot);
    VQ_CUDA(cudaMemcpyAsync(w, host.data(), sizeof(BatchInst) * (size_t)count, cudaMemcpyHostToDevice, st));
    VQ_CUDA(cudaMemcpyAsync(w + ib, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice, st));
    VQ_CUDA(cudaMemcpyAsync(w + ib + ob, begin.data(), sizeof(int32_t) * begin.size(), cudaMemcpyHostToDevice, st));
    uint8_t* wr = w + ib + ob + bb;
    VQ_CUDA(cudaMemcpyAsync(wr, rd.data(), sizeof(ReadInst) * (size_t)count, cudaMemcpyHostToDevice, st));
    uint8_t* wl[4];
    {
        uint8_t* at = wr + rb;
        for (int t = 0; t < 4; ++t) {
            wl[t] = at;
            if (!rwork[t].empty())
                VQ_CUDA(cudaMemcpyAsync(at, rwork[t].data(), sizeof(int32_t) * rwork[t].size(),
                                        cudaMemcpyHostToDevice, st));
            at += wb[t];
        }
    }
    VQ_CUDA(cudaMemcpyAsync(seed_dev, &seed, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    BatchArgs a;
    a.inst = reinterpret_cast<const BatchInst*>(w);
    a.order = reinterpret_cast<const int32_t*>(w + ib);
    a.cta_begin = reinterpret_cast<const int32_t*>(w + ib + ob);
    a.R = R;
    a.G = split;
    a.RG = RG;
    a.K = p.K;
    a.dt = p.dt;
    a.a0 = p.a0;
    a.sigma0 = p.sigma0;
    a.seed = seed_dev;
    a.a_table = ctxs[0]->a_table.as<float>();
    a.err = d_err;
    a.alpha = p.alpha;
    const ReadInst* rdev = reinterpret_cast<const ReadInst*>(wr);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (graph) {
        if (!graph->e0) VQ_CUDA(cudaEventCreate(&graph->e0));
        if (!graph->e1) VQ_CUDA(cudaEventCreate(&graph->e1));
        e0 = graph->e0;
        e1 = graph->e1;
    } else {
        VQ_CUDA(cudaEventCreate(&e0));
        VQ_CUDA(cudaEventCreate(&e1));
    }
    // the device part of the solve: operand padding, the persistent kernel
    // between two timing events, and the final readout (one energy launch per
    // element type of Q in the batch, one finish launch)
    auto enqueue = [&]() -> int {
        const unsigned flags = graph ? cudaEventRecordExternal : cudaEventRecordDefault;
        for (const auto& z : zero) VQ_CUDA(cudaMemsetAsync(z.first, 0, z.second, st));
        VQ_CUDA(cudaEventRecordWithFlags(e0, st, flags));
        fn<<<ctas, stages == 6 ? batch_threads<6>() : batch_threads<4>(), smem, st>>>(a);
        VQ_LAUNCH_CHECK("batch kernel");
        VQ_CUDA(cudaEventRecordWithFlags(e1, st, flags));
        for (int t = 0; t < 4; ++t) {
            const unsigned blocks = (unsigned)(rwork[t].size() / 2);
            if (!blocks) continue;
            const int32_t* wd = reinterpret_cast<const int32_t*>(wl[t]);
            switch (t) {
                case VELOXQ_I8: k_batch_energy<int8_t><<<blocks, 256, 0, st>>>(rdev, wd, R); break;
                case VELOXQ_I32: k_batch_energy<int32_t><<<blocks, 256, 0, st>>>(rdev, wd, R); break;
                case VELOXQ_F32: k_batch_energy<float><<<blocks, 256, 0, st>>>(rdev, wd, R); break;
                default: k_batch_energy<double><<<blocks, 256, 0, st>>>(rdev, wd, R); break;
            }
        }
        k_batch_finish<<<(unsigned)count, 256, 0, st>>>(rdev, R, d_best_all);
        VQ_LAUNCH_CHECK("batch readout");
        return VELOXQ_OK;
    };
    for (int t = 0; t < 4; ++t) nl += rwork[t].empty() ? 0 : 1;
    nl += 2;   // the batched kernel and the finish
    if (launches) *launches = nl;
    if (!graph) {
        VQ_TRY(enqueue());
    } else {
        // one graph per kind of launch: everything the captured nodes bake in
        std::vector<uint64_t> key = {(uint64_t)(uintptr_t)fn, (uint64_t)ctas, (uint64_t)smem, (uint64_t)(uintptr_t)w,
                                     (uint64_t)(uintptr_t)d_best_all, (uint64_t)(uintptr_t)d_err, (uint64_t)R,
                                     (uint64_t)split, (uint64_t)p.K, (uint64_t)count,
                                     (uint64_t)(uintptr_t)a.a_table};
        for (float f : {p.dt, p.a0, p.sigma0, p.alpha}) {
            uint32_t u;
            std::memcpy(&u, &f, 4);
            key.push_back(u);
        }
        for (int t = 0; t < 4; ++t) key.push_back(rwork[t].size());
        for (const auto& z : zero) {
            key.push_back((uint64_t)(uintptr_t)z.first);
            key.push_back(z.second);
        }
        if (!graph->exec || graph->key != key) {
            if (graph->exec) {
                cudaGraphExecDestroy(graph->exec);
                graph->exec = nullptr;
            }
            cudaGraph_t g = nullptr;
            VQ_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            const int rc = enqueue();
            const cudaError_t ce = cudaStreamEndCapture(st, &g);
            if (rc != VELOXQ_OK) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (ce != cudaSuccess) return cuda_fail(ce, "batch graph capture");
            const cudaError_t ie = cudaGraphInstantiate(&graph->exec, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) {
                graph->exec = nullptr;
                return cuda_fail(ie, "batch graph instantiate");
            }
            graph->key = key;
        }
        VQ_CUDA(cudaGraphLaunch(graph->exec, st));
    }
    VQ_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    VQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms_main) *ms_main = ms;
    if (!graph) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    return VELOXQ_OK;
}

}  // namespace vq
