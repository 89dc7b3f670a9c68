// vq_tc.cu -- dense local field F = Qoff S on the 5th-generation tensor cores
// (tcgen05, accumulators in tensor memory), operands staged by TMA, with the
// ballistic-SB update fused into the epilogue.
//
// D[i][r] = sum_j Qop[i][j] Sop[r][j]: M = variables (rows of Qoff), N =
// replicas, K = variables. Both operands are K-major (Qoff row-major, S
// replica-major), 128-byte K blocks with the 128-byte swizzle.
// CTA pairs (clusters of 2, tcgen05 cta_group::2): a pair computes a
// 256 x 256 tile with M = 256 MMAs issued by the even CTA. Each CTA stages
// its own 128 rows of Qoff and its own 128 replicas of S; each CTA's tensor
// memory holds the accumulator of its 128 rows for all 256 replicas.
//   BF16: Qop = bf16(Qoff), Sop = bf16(s)                (kind::f16)
//   FP8 : Qop = e4m3(Qoff_ij / q_i), q_i = amax_i / 448  (kind::f8f6f4)
//         S in two E4M3 terms of the same scale (TERMS = 2):
//           v = 448 s (|s| <= 1 by the walls), hi = e4m3(v), lo = e4m3(v - hi)
//         (v - hi is exact in FP32), so S carries about 7 significant bits
//         and the product's error is that of Q's rounding alone; both terms
//         are multiplied by the same Qop tile and accumulate into the same
//         FP32 accumulator, acc = Qop hi + Qop lo.
//         One term (TERMS = 1): Sop = hi only (VELOXQ_PREC_FP8_ONE_TERM, and
//         Parallel Annealing, whose operand +-448 is exact so lo = 0).
//         F_i = acc q_i / 448
// A stage is 32 KB per CTA with one S term (6 stages in flight) and 48 KB
// with two (4 stages); both fill 192 KB of shared memory.
// The kernel is persistent: one CTA per SM, the pairs walk the pair tiles
// t = pair, + pairs, ...; two accumulator buffers in tensor memory let the
// epilogue of one tile overlap the main loop of the next.
// Warp roles: warp 0 issues TMA (both CTAs; completion is counted on the
// even CTA's barrier), warp 1 allocates tensor memory (both CTAs) and issues
// the MMAs (even CTA), warps 2-9 read the accumulator tile (a 32-lane quarter
// and half of the columns each) and run the update for their rows. Every
// wait is bounded: on timeout the kernel records a code in the error word
// and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstdlib>

#include "vq_internal.cuh"

namespace vq {

namespace {

// BM rows per CTA (2 BM per pair), BN replicas per pair (BN / 2 staged per CTA)
constexpr int BM = 128, BN = 256, BNH = BN / 2, BKB = 128;
constexpr uint32_t A_BYTES = BM * BKB, B_BYTES = BNH * BKB;
// a stage holds the Qop block and TERMS blocks of Sop
template <int TERMS> constexpr uint32_t stage_bytes() { return A_BYTES + TERMS * B_BYTES; }
template <int TERMS> constexpr int stages_of() { return TERMS == 2 ? 4 : 6; }
constexpr uint32_t PIPE_BYTES = 6 * stage_bytes<1>();
static_assert(stages_of<2>() * stage_bytes<2>() == PIPE_BYTES, "both stage forms fill the same 192 KB");
constexpr size_t TC_SMEM = (size_t)PIPE_BYTES + 1024 /*align*/ + 256 /*barriers, tensor-memory slot*/;
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz

enum { TC_ERR_PRODUCER = 1, TC_ERR_MMA = 2, TC_ERR_EPILOGUE = 4, TC_ERR_SELFTEST = 8, TC_ERR_DEPEND = 16 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// The same with cluster-scope acquire, for barriers the peer CTA arrives on.
__device__ __forceinline__ bool mbar_try_wait_cl(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false (and the error word set) if the phase does not complete
// within the budget or another thread already gave up.
template <bool CLUSTER = false>
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code,
                                          long long budget = kWaitCycles) {
    const long long t0 = clock64();
    uint32_t spins = 0;
    while (!(CLUSTER ? mbar_try_wait_cl(bar, parity) : mbar_try_wait(bar, parity))) {
        if ((++spins & 1023u) == 0) {
            if (*(volatile int*)err) return false;
            if (clock64() - t0 > budget) {
                atomicOr(err, code);
                return false;
            }
        }
    }
    return true;
}

// ---- cluster of two CTAs ----
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// shared::cluster address of the same shared variable in CTA `rank`
__device__ __forceinline__ uint32_t mapa(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cl_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cl_addr) : "memory");
}

// 2-D tile load into this CTA's shared memory; completion is counted on the
// barrier at cluster address `bar_cl` (the even CTA's barrier of the pair).
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, int x, int y, uint32_t bar_cl) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2 "
        "[%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar_cl)
        : "memory");
}
// The same with an L2 cache policy (the coupling operand, which every column
// block of every step reads again, is kept in L2 ahead of streaming data).
__device__ __forceinline__ void tma_load_2d_pair_hint(void* dst, const CUtensorMap* map, int x, int y,
                                                      uint32_t bar_cl, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2.L2::cache_hint "
        "[%0], [%1, {%2, %3}], [%4], %5;"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar_cl), "l"(pol)
        : "memory");
}
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// ---- completion counters between CTAs of one grid (steps of a run) ----
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(uint32_t* p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Generic-proxy writes to global memory made visible to (and ordered with)
// the async proxy: the bulk tensor copies of another CTA read them.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
// Bounded wait until *c >= target: false (and the error word set) if it is
// not reached within the budget or another thread already gave up.
__device__ __forceinline__ bool count_wait(const uint32_t* c, uint32_t target, int* err, int code) {
    const long long t0 = clock64();
    uint32_t spins = 0;
    while (ld_acquire_u32(c) < target) {
        if ((++spins & 255u) == 0) {
            if (*(volatile int*)err) return false;
            if (clock64() - t0 > kWaitCycles) {
                atomicOr(err, code);
                return false;
            }
        }
    }
    return true;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Tensor memory of a CTA pair: one warp of each CTA allocates (and frees)
// together; both CTAs receive the same column address.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// core groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
    const uint32_t a = smem_u32(p);
    uint64_t d = 0;
    d |= (uint64_t)((a & 0x3FFFFu) >> 4);          // start address
    d |= (uint64_t)1 << 16;                         // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset
    d |= (uint64_t)1 << 46;                         // descriptor version
    d |= (uint64_t)2 << 61;                         // 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulator, A/B format, K-major, N, M (the
// pair's M = 2 BM).
template <int PREC> __host__ __device__ constexpr uint32_t instr_desc() {
    return (1u << 4)                                   // D format F32
           | ((PREC == 1 ? 1u : 0u) << 7)              // A: BF16 (f16 kind) / E4M3 (f8f6f4 kind)
           | ((PREC == 1 ? 1u : 0u) << 10)             // B: same
           | ((uint32_t)(BN >> 3) << 17)               // N
           | ((uint32_t)((2 * BM) >> 4) << 24);        // M
}

// M = 256 MMA of the pair, issued by the even CTA: A rows from both CTAs'
// shared memory, B (replicas) likewise, the accumulator in both CTAs'
// tensor memory.
template <int PREC>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
    if constexpr (PREC == 1) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
            ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accum)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n"
            ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accum)
            : "memory");
    }
}
// Arrive on the barrier at the same offset in both CTAs once the MMAs issued
// so far have completed.
__device__ __forceinline__ void umma_commit_pair(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .b16 m;\n\tmov.b16 m, 3;\n\t"
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], m;\n\t}\n"
        ::"r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TcArgs {
    int32_t n, R, n_pad;
    int32_t k, k_end;        // steps k .. k_end - 1 of the schedule (one launch)
    float dt, a0, c0;
    const float* S_a;        // [R][n] fp32 state of the first step (even steps of the run read it)
    float* S_b;              // [R][n] the other state buffer (null: field only)
    float* Y;                // [R][n]
    void* sop[2];            // [R][n_pad] per term: operand buffers; the first step reads sop[cur]
    int32_t cur;
    int32_t colmajor;        // runs of several steps: tiles of a step in groups of this many replica
                             // column blocks, row block by row block within a group; 0: row-major
    const float* bf;         // [n]
    const float* qscale;     // [n] FP8 row scales (FP8 only)
    const float* a_table;
    float* F_out;            // [R][n] field of the last step, or null
    int* err;
    float alpha;             // PA momentum
    int64_t plane;           // elements from the hi plane of an operand buffer to its lo plane (two S terms)
    uint32_t* done;          // [NT] epilogue warps finished per replica column block (zeroed per launch)
};

// Operand of s: bf16(s); or v = 448 s as hi = e4m3(v) and, with two terms,
// lo = e4m3(v - hi) at idx + plane (v - hi is exact in FP32).
template <int PREC, int TERMS>
__device__ __forceinline__ void store_op(void* base, int64_t idx, int64_t plane, float s) {
    if constexpr (PREC == 1) {
        reinterpret_cast<__nv_bfloat16*>(base)[idx] = __float2bfloat16_rn(s);
    } else {
        __nv_fp8_storage_t* o = reinterpret_cast<__nv_fp8_storage_t*>(base);
        const float v = __fmul_rn(448.0f, s);
        const __nv_fp8_storage_t hi = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
        o[idx] = hi;
        if constexpr (TERMS == 2) {
            const float hf = __half2float(__half(__nv_cvt_fp8_to_halfraw(hi, __NV_E4M3)));
            o[idx + plane] = __nv_cvt_float_to_fp8(__fsub_rn(v, hf), __NV_SATFINITE, __NV_E4M3);
        }
    }
}

// One launch runs steps k .. k_end - 1. The pairs walk the pair tiles of all
// those steps, g = pair, pair + pairs, ... with g = j * tiles + t for step
// k + j. A step's tile (row block r, replica column block c) reads the
// operand of column block c over every variable, which the previous step's
// tiles (all r, same c) write: with colmajor = G, a step's tiles come in
// groups of G column blocks (t = c0 MT + r gc + (c - c0) within the group
// [c0, c0 + gc)), so a step's first group is ready as soon as the previous
// step's is, and pairs flow from one step into the next without a
// grid-wide barrier, while the column blocks of a group share each Qoff row
// block in L2. The
// dependency is counted per column block: every epilogue warp adds 1 to
// done[c] (release) once its rows and columns of the tile are written; a
// tile of step j > 0 starts loading the operand (and the epilogue reads its
// state) only after done[c] >= 16 MT j (acquire), i.e. when the whole column
// block of every earlier step of the launch is written. That also orders the
// reuse of the ping-pong buffers: what a tile overwrites was last read by the
// previous step's tiles of the same column block. A pair only ever waits for
// tiles with a lower g, all CTAs of the grid are resident (one per SM, at
// most the co-resident clusters), and every wait is bounded.
// One step (k_end = k + 1) is the plain fused step (row-major tiles, odd
// steps walked backwards so that a step starts on the state the previous
// one wrote last).
// METHOD: the integrator (veloxq_method), a template parameter so that each
// form keeps its own register allocation. TERMS: S operand terms (1, or 2 for
// FP8 hi + lo; tmL* map the lo planes, unused with one term).
template <int PREC, int TERMS, bool FIELD_ONLY, int METHOD>
__global__ void __launch_bounds__(320, 1) k_tc_step(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB0,
                                                    const __grid_constant__ CUtensorMap tmB1,
                                                    const __grid_constant__ CUtensorMap tmL0,
                                                    const __grid_constant__ CUtensorMap tmL1, const TcArgs a) {
    constexpr int STAGES = stages_of<TERMS>();
    constexpr uint32_t STAGE_BYTES = stage_bytes<TERMS>();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);   // even CTA: both stages landed
    uint64_t* empty = full + STAGES;      // both CTAs: stage consumed by the MMAs
    uint64_t* accf = empty + STAGES;      // [2] both CTAs: accumulator buffer ready for the epilogue
    uint64_t* acce = accf + 2;            // [2] even CTA: buffer drained by both CTAs' epilogues
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int pair = blockIdx.x >> 1, pairs = gridDim.x >> 1;
    constexpr int EB = PREC == 1 ? 2 : 1;
    constexpr int BK = BKB / EB;                 // elements per K block
    constexpr int KSTEP_B = 32;                  // bytes of K per MMA (16 bf16 / 32 e4m3)
    const int num_kb = (a.n_pad + BK - 1) / BK;
    const int MT = (a.n + 2 * BM - 1) / (2 * BM), NT = (a.R + BN - 1) / BN;
    const int tiles = MT * NT;
    const int steps = a.k_end - a.k;
    const int64_t work = (int64_t)steps * tiles;
    const uint32_t per_col = 16u * (uint32_t)MT;   // epilogue warps of one column block of one step
    // tile t of step j: row block r, column block c
    auto tile_rc = [&](int j, int t, int& r, int& c) {
        if (a.colmajor) {
            // group of G column blocks [c0, c0 + gc): every row block of
            // the group, its column blocks next to each other (they read
            // the same Qoff row block at about the same time)
            const int G = a.colmajor;
            const int c0 = (t / (G * MT)) * G;
            const int gc = min(G, NT - c0);
            const int u = t - c0 * MT;
            r = u / gc;
            c = c0 + (u - r * gc);
        } else {
            const int tt2 = ((a.k + j) & 1) ? tiles - 1 - t : t;
            r = tt2 / NT;
            c = tt2 - r * NT;
        }
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 16);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, 2 * BN);
    tc_fence_before();
    cluster_sync();                              // both CTAs' barriers exist before any remote arrive
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // Programmatic dependent launch: everything above (barriers, tensor
    // memory, the cluster handshake) may overlap the previous kernel on the
    // stream; nothing it wrote is read before this wait returns. The next
    // kernel may then be scheduled, onto SMs this grid frees as it exits
    // (every CTA of this grid is resident by now, one per SM).
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    if (warp == 0) {
        if (lane == 0) {
            const uint64_t qpol = l2_evict_last_policy();
            uint32_t it = 0;
            bool ok = true;
            for (int64_t g = pair; g < work && ok; g += pairs) {
                const int j = (int)(g / tiles), t = (int)(g - (int64_t)j * tiles);
                int r, c;
                tile_rc(j, t, r, c);
                const int m0 = r * (2 * BM) + (int)rank * BM, n0 = c * BN + (int)rank * BNH;
                // the previous steps' column block c: every operand block this tile reads
                if (j > 0) {
                    if (!count_wait(a.done + c, per_col * (uint32_t)j, a.err, TC_ERR_DEPEND)) break;
                    fence_proxy_async_global();
                }
                const int buf = (a.cur + j) & 1;
                const CUtensorMap* mb = buf ? &tmB1 : &tmB0;
                const CUtensorMap* ml = buf ? &tmL1 : &tmL0;
                for (int kb = 0; kb < num_kb; ++kb) {
                    const uint32_t s = it % STAGES, u = it / STAGES;
                    if (u > 0 && !mbar_wait<true>(&empty[s], (u - 1) & 1, a.err, TC_ERR_PRODUCER)) { ok = false; break; }
                    uint8_t* sa = smem + s * STAGE_BYTES;
                    if (leader) mbar_expect_tx(&full[s], 2 * STAGE_BYTES);
                    const uint32_t fb = mapa(smem_u32(&full[s]), 0);
                    tma_load_2d_pair_hint(sa, &tmA, kb * BK, m0, fb, qpol);
                    tma_load_2d_pair(sa + A_BYTES, mb, kb * BK, n0, fb);
                    if constexpr (TERMS == 2) tma_load_2d_pair(sa + A_BYTES + B_BYTES, ml, kb * BK, n0, fb);
                    ++it;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            constexpr uint32_t idesc = instr_desc<PREC>();
            uint32_t it = 0, tt = 0;
            bool ok = true;
            for (int64_t g = pair; g < work && ok; g += pairs, ++tt) {
                const uint32_t b = tt & 1u;
                if (tt >= 2 && !mbar_wait<true>(&acce[b], ((tt >> 1) - 1) & 1u, a.err, TC_ERR_MMA)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d = tmem + b * BN;
                for (int kb = 0; kb < num_kb; ++kb) {
                    const uint32_t s = it % STAGES, u = it / STAGES;
                    if (!mbar_wait<true>(&full[s], u & 1, a.err, TC_ERR_MMA)) { ok = false; break; }
                    tc_fence_after();
                    const uint8_t* sa = smem + s * STAGE_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BKB / KSTEP_B; ++kk) {
                        const uint64_t da = smem_desc(sa + kk * KSTEP_B);
                        umma<PREC>(d, da, smem_desc(sa + A_BYTES + kk * KSTEP_B), idesc, (kb | kk) != 0 ? 1u : 0u);
                        // the lo term of S against the same Qop slice, into the same accumulator
                        if constexpr (TERMS == 2)
                            umma<PREC>(d, da, smem_desc(sa + A_BYTES + B_BYTES + kk * KSTEP_B), idesc, 1u);
                    }
                    umma_commit_pair(&empty[s]);
                    ++it;
                }
                if (ok) umma_commit_pair(&accf[b]);
            }
        }
    } else {
        // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. +31 (this
        // CTA's rows); the first four epilogue warps take replica columns
        // [0, BN/2), the next four the rest
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;
        const uint32_t acce_cl = mapa(smem_u32(&acce[0]), 0);
        constexpr int CW = 16;   // columns per tensor-memory load
        const int c_begin = half * (BN / (2 * CW)), c_end = c_begin + BN / (2 * CW);   // 8 chunks, even
        uint32_t tt = 0;
        for (int64_t g = pair; g < work; g += pairs, ++tt) {
            const uint32_t b = tt & 1u;
            const int j = (int)(g / tiles), t = (int)(g - (int64_t)j * tiles);
            int r, c;
            tile_rc(j, t, r, c);
            const int k = a.k + j;
            const float a_k = FIELD_ONLY ? 0.0f : __ldg(a.a_table + k);
            const float lam = (FIELD_ONLY || METHOD != vqd::METHOD_PA) ? 0.0f : vqd::pa_lambda(a_k, a.a0);
            const float* S_cur = (j & 1) ? a.S_b : a.S_a;
            float* S_nxt = (j & 1) ? const_cast<float*>(a.S_a) : a.S_b;
            void* sop_nxt = a.sop[(a.cur + j + 1) & 1];
            float* F_out = j == steps - 1 ? a.F_out : nullptr;
            const int m0 = r * (2 * BM) + (int)rank * BM, n0 = c * BN;
            const int row = m0 + q * 32 + lane;
            const bool row_ok = row < a.n;
            float fscale = 1.0f, bi = 0.0f;
            if (row_ok) {
                if constexpr (PREC == 2) fscale = __ldg(a.qscale + row) * (1.0f / 448.0f);
                if constexpr (!FIELD_ONLY) bi = __ldg(a.bf + row);
            }
            // the state of these rows was written by the previous step's tile
            if (j > 0) {
                bool got = false;
                if (lane == 0) got = count_wait(a.done + c, per_col * (uint32_t)j, a.err, TC_ERR_DEPEND);
                if (__shfl_sync(0xffffffffu, got ? 1 : 0, 0) == 0) break;
                (void)ld_acquire_u32(a.done + c);
            }
            // Positions and momenta of a chunk: loaded one chunk ahead of its
            // use (the first before the accumulator is ready), so two chunks'
            // loads are in flight while one is updated. They are read once per
            // step and kept out of L2's way (evict-first).
            float sv0[CW], yv0[CW], sv1[CW], yv1[CW];
            auto load_chunk = [&](int cc, float (&sv)[CW], float (&yv)[CW]) {
                if constexpr (!FIELD_ONLY) {
                    const int r0 = n0 + cc * CW;
#pragma unroll
                    for (int jj = 0; jj < CW; ++jj) {
                        const bool ok = row_ok && r0 + jj < a.R;
                        const int64_t p = (int64_t)(r0 + jj) * a.n + row;
                        sv[jj] = ok ? __ldcs(S_cur + p) : 0.0f;
                        yv[jj] = ok ? __ldcs(a.Y + p) : 0.0f;
                    }
                }
            };
            auto update_chunk = [&](int cc, const float (&sv)[CW], const float (&yv)[CW]) {
                uint32_t v[CW];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + b * BN + (uint32_t)(cc * CW), v);
                const int r0 = n0 + cc * CW;
#pragma unroll
                for (int jj = 0; jj < CW; ++jj) {
                    const bool ok = row_ok && r0 + jj < a.R;
                    const int64_t p = (int64_t)(r0 + jj) * a.n + row;
                    const float F = __uint_as_float(v[jj]) * fscale;
                    if (ok && F_out) F_out[p] = F;
                    if constexpr (!FIELD_ONLY) {
                        float s = sv[jj], y = yv[jj];
                        if constexpr (METHOD == vqd::METHOD_PA) vqd::pa_update(F, bi, lam, a.dt, a.alpha, a.c0, s, y);
                        else if constexpr (METHOD == vqd::METHOD_ASB) vqd::asb_update(F, bi, a_k, a.dt, a.a0, a.c0, s, y);
                        else vqd::bsb_update(F, bi, a_k, a.dt, a.a0, a.c0, s, y);
                        if (ok) {
                            __stcs(S_nxt + p, s);
                            __stcs(a.Y + p, y);
                            store_op<PREC, TERMS>(sop_nxt, (int64_t)(r0 + jj) * a.n_pad + row, a.plane,
                                                  METHOD == vqd::METHOD_PA ? vqd::pa_sign(s) : s);
                        }
                    }
                }
            };
            load_chunk(c_begin, sv0, yv0);
            if (!mbar_wait<true>(&accf[b], (tt >> 1) & 1u, a.err, TC_ERR_EPILOGUE)) break;
            tc_fence_after();
#pragma unroll 1
            for (int cc = c_begin; cc < c_end; cc += 2) {
                load_chunk(cc + 1, sv1, yv1);
                update_chunk(cc, sv0, yv0);
                if (cc + 2 < c_end) load_chunk(cc + 2, sv0, yv0);
                update_chunk(cc + 1, sv1, yv1);
            }
            // hand the accumulator buffer back to the even CTA's MMA thread,
            // and count this warp's part of the tile as written (for the
            // bulk copies and loads of the next step's tiles)
            if (steps > 1) {
                fence_proxy_async_global();
                __threadfence();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive_remote(acce_cl + b * 8);
                if (steps > 1) red_release_add(a.done + c, 1u);
            }
        }
    }
    // neither CTA leaves while the other may still read its shared memory or
    // arrive on its barriers
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, 2 * BN);
}

// The bounded wait of the kernels above on a barrier that nothing arrives on:
// it runs out after `budget` cycles, records its code in the error word and
// returns (the path every kernel takes when a wait gives up).
__global__ void k_wait_selftest(int* err, long long budget) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&bar, 0, err, TC_ERR_SELFTEST, budget);
    __syncthreads();
}

// ---- operand preparation --------------------------------------------------
__global__ void k_quant_q_bf16(int64_t n, int64_t n_pad, const float* __restrict__ q, __nv_bfloat16* out) {
    const int64_t i = blockIdx.x;
    for (int64_t j = threadIdx.x; j < n_pad; j += blockDim.x)
        out[i * n_pad + j] = __float2bfloat16_rn(j < n ? q[i * n + j] : 0.0f);
}

// per-row scale q_i = amax_i / 448 (1 for an all-zero row), e4m3(Qoff_ij / q_i)
__global__ void k_quant_q_fp8(int64_t n, int64_t n_pad, const float* __restrict__ q, __nv_fp8_storage_t* out,
                              float* scale) {
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
    const float amax = sh[0];
    const float sc = amax > 0.0f ? amax / 448.0f : 1.0f;
    const float inv = 1.0f / sc;
    for (int64_t j = threadIdx.x; j < n_pad; j += blockDim.x)
        out[i * n_pad + j] = __nv_cvt_float_to_fp8(j < n ? q[i * n + j] * inv : 0.0f, __NV_SATFINITE, __NV_E4M3);
    if (threadIdx.x == 0) scale[i] = sc;
}

template <int PREC, int TERMS>
__global__ void k_quant_s(int64_t R, int64_t n, int64_t n_pad, const float* __restrict__ S, void* out, int method) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= R * n_pad) return;
    const int64_t r = t / n_pad, j = t - r * n_pad;
    store_op<PREC, TERMS>(out, t, R * n_pad, j < n ? vqd::field_operand(method, S[r * n + j]) : 0.0f);
}

// ---- tensor maps ------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D K-major operand [rows][n_pad], box {128 bytes of K, box_rows}
int make_map(CUtensorMap* m, void* base, int prec, int64_t rows, int64_t n_pad, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return fail(VELOXQ_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    const int eb = prec == 1 ? 2 : 1;
    cuuint64_t dims[2] = {(cuuint64_t)n_pad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(n_pad * eb)};
    cuuint32_t box[2] = {(cuuint32_t)(BKB / eb), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, prec == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(VELOXQ_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return VELOXQ_OK;
}

}  // namespace

int64_t tc_pad(int64_t n) { return (n + 15) / 16 * 16; }

// S operand terms: two E4M3 terms for FP8 (hi + lo), one for FP8_ONE_TERM,
// BF16, and for Parallel Annealing, whose operand +-1 is exact in one term.
int tc_terms(int prec, int method) {
    return prec == VELOXQ_PREC_FP8 && method != VELOXQ_METHOD_PA ? 2 : 1;
}

// Quantise Qoff once per precision (kept in the context).
int tc_prepare_q(veloxq_ctx* ctx, int prec) {
    const int64_t n = ctx->n, np = tc_pad(n);
    cudaStream_t st = ctx->stream;
    if (prec == VELOXQ_PREC_BF16) {
        if (!ctx->qoff16.p) {
            VQ_TRY(ctx->qoff16.ensure(sizeof(__nv_bfloat16) * (size_t)(n * np)));
            k_quant_q_bf16<<<(unsigned)n, 256, 0, st>>>(n, np, ctx->qoff32.as<float>(), ctx->qoff16.as<__nv_bfloat16>());
        }
    } else {
        if (!ctx->qoff8.p) {
            VQ_TRY(ctx->qoff8.ensure((size_t)(n * np)));
            VQ_TRY(ctx->qscale8.ensure(sizeof(float) * (size_t)n));
            k_quant_q_fp8<<<(unsigned)n, 256, 0, st>>>(n, np, ctx->qoff32.as<float>(), ctx->qoff8.as<__nv_fp8_storage_t>(),
                                                       ctx->qscale8.as<float>());
        }
    }
    VQ_LAUNCH_CHECK("tc quantize Q");
    return VELOXQ_OK;
}

// Tensor maps for Q and for the two S operand buffers (each R x n_pad per
// term; with two terms the lo plane follows the hi plane, and ms*_lo map it).
int tc_maps(veloxq_ctx* ctx, int prec, int terms, int32_t R, void* sop0, void* sop1, CUtensorMap* mq,
            CUtensorMap* ms0, CUtensorMap* ms1, CUtensorMap* ms0_lo, CUtensorMap* ms1_lo) {
    const int64_t n = ctx->n, np = tc_pad(n);
    void* qb = prec == VELOXQ_PREC_BF16 ? ctx->qoff16.p : ctx->qoff8.p;
    VQ_TRY(make_map(mq, qb, prec, n, np, BM));
    const size_t plane = (size_t)R * (size_t)np * (prec == VELOXQ_PREC_BF16 ? 2 : 1);
    VQ_TRY(make_map(ms0, sop0, prec, R, np, BNH));
    if (terms == 2) VQ_TRY(make_map(ms0_lo, static_cast<uint8_t*>(sop0) + plane, prec, R, np, BNH));
    if (sop1) {
        VQ_TRY(make_map(ms1, sop1, prec, R, np, BNH));
        if (terms == 2) VQ_TRY(make_map(ms1_lo, static_cast<uint8_t*>(sop1) + plane, prec, R, np, BNH));
    }
    return VELOXQ_OK;
}

int tc_quant_s(veloxq_ctx* ctx, int prec, int32_t R, const float* S, void* sop, const Rule& rule) {
    const int64_t n = ctx->n, np = tc_pad(n);
    const int64_t total = (int64_t)R * np;
    const unsigned blocks = (unsigned)div_up(total, 256);
    if (prec == VELOXQ_PREC_BF16)
        k_quant_s<1, 1><<<blocks, 256, 0, ctx->stream>>>(R, n, np, S, sop, rule.method);
    else if (tc_terms(prec, rule.method) == 2)
        k_quant_s<2, 2><<<blocks, 256, 0, ctx->stream>>>(R, n, np, S, sop, rule.method);
    else
        k_quant_s<2, 1><<<blocks, 256, 0, ctx->stream>>>(R, n, np, S, sop, rule.method);
    VQ_LAUNCH_CHECK("tc quantize S");
    return VELOXQ_OK;
}

// A K-major operand map of the field kernel: A (rows of the coupling
// matrix, box of BM rows) or B (replicas, box of BN/2 rows).
int tc_operand_map(CUtensorMap* m, void* base, int prec, int64_t rows, int64_t n_pad, bool a_operand) {
    return make_map(m, base, prec, rows, n_pad, a_operand ? BM : BNH);
}

int tc_wait_selftest(long long budget, int* code_out) {
    int* err = nullptr;
    VQ_CUDA(cudaMalloc(&err, sizeof(int)));
    int h = 0;
    cudaError_t e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32>>>(err, budget);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
    *code_out = h;
    return VELOXQ_OK;
}

size_t tc_sop_bytes(veloxq_ctx* ctx, int prec, int terms, int32_t R) {
    return (size_t)terms * (size_t)R * (size_t)tc_pad(ctx->n) * (prec == VELOXQ_PREC_BF16 ? 2 : 1);
}

namespace {
using TcKernel = void (*)(const CUtensorMap, const CUtensorMap, const CUtensorMap, const CUtensorMap,
                          const CUtensorMap, const TcArgs);

template <int PREC, int TERMS> TcKernel pick_kernel(bool field_only, int method) {
    if (field_only) return k_tc_step<PREC, TERMS, true, 0>;
    if (method == VELOXQ_METHOD_PA) return k_tc_step<PREC, TERMS, false, vqd::METHOD_PA>;
    if (method == VELOXQ_METHOD_ASB) return k_tc_step<PREC, TERMS, false, vqd::METHOD_ASB>;
    return k_tc_step<PREC, TERMS, false, vqd::METHOD_BSB>;
}

// co-resident CTA pairs of the step kernel, per device
constexpr int kMaxDevices = 64;
int g_max_pairs[kMaxDevices];

// Steps per launch at most: the completion counters (16 MT per column block
// and step) stay far below 2^32.
constexpr int kMaxRunSteps = 4096;

// Replica column blocks per group of a multi-step run's tile order. One
// block at a time lets the next step start after a quarter of this one (at
// R = 1024) but reads Qoff once per column block; groups of two read it
// half as often. Measured at SK n = 8192, R = 1024 (us per step, groups of
// 1 / 2 / 4): BF16 82.5 / 80.0 / 98.0, FP8 one term 51.8 / 51.1 / 66.0, FP8
// two terms (tensor-bound) 69.9 / 70.7 / 92.2. VELOXQ_TC_COLGROUP (1 to 16)
// fixes it.
int tc_column_group(int prec, int terms) {
    static const int forced = [] {
        const char* e = std::getenv("VELOXQ_TC_COLGROUP");
        const int v = e ? std::atoi(e) : 0;
        return (v >= 1 && v <= 16) ? v : 0;
    }();
    if (forced) return forced;
    return (prec == VELOXQ_PREC_FP8 && terms == 2) ? 1 : 2;
}
}  // namespace

int tc_run(veloxq_ctx* ctx, int prec, int32_t R, const CUtensorMap& mq, const CUtensorMap* ms,
           const CUtensorMap* ms_lo, int cur, const float* S_a, float* S_b, float* Y, void* const* sop,
           const float* a_table, int k_begin, int k_end, float dt, float a0, float c0, float* F_out, int* err,
           const Rule& rule) {
    const bool field_only = S_b == nullptr;
    if (k_end <= k_begin) return VELOXQ_OK;
    if (field_only && k_end != k_begin + 1) return fail(VELOXQ_EINVAL, "the field alone is one step");
    // the field alone takes s itself as the operand
    const int terms = tc_terms(prec, field_only ? VELOXQ_METHOD_BSB : rule.method);
    if (terms == 2 && !ms_lo) return fail(VELOXQ_EINVAL, "two-term FP8 operand without its lo-plane maps");
    if (ctx->device < 0 || ctx->device >= kMaxDevices) return fail(VELOXQ_EUNSUPPORTED, "device ordinal out of range");
    const int sms = device_sms(ctx->device);
    const int64_t MT = div_up(ctx->n, 2 * BM), NT = div_up(R, BN), tiles = MT * NT;
    TcKernel fn;
    if (prec == VELOXQ_PREC_BF16) fn = pick_kernel<1, 1>(field_only, rule.method);
    else if (terms == 2) fn = pick_kernel<2, 2>(field_only, rule.method);
    else fn = pick_kernel<2, 1>(field_only, rule.method);
    VQ_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(320);
    cfg.dynamicSmemBytes = TC_SMEM;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // as many pairs as can be resident at once (one CTA per SM; every form
    // has the same block size and shared memory)
    int& max_pairs = g_max_pairs[ctx->device];
    if (!max_pairs) {
        cfg.gridDim = dim3((unsigned)(sms & ~1));
        int c = 0;
        if (cudaOccupancyMaxActiveClusters(&c, fn, &cfg) != cudaSuccess || c < 1) {
            cudaGetLastError();
            c = sms / 2;
        }
        max_pairs = std::max(1, std::min(c, sms / 2));
    }
    const CUtensorMap& lo0 = terms == 2 ? ms_lo[0] : ms[0];
    const CUtensorMap& lo1 = terms == 2 ? ms_lo[1] : ms[1];
    for (int k0 = k_begin; k0 < k_end; k0 += kMaxRunSteps) {
        const int k1 = std::min(k_end, k0 + kMaxRunSteps);
        const int steps = k1 - k0;
        TcArgs a;
        a.n = (int32_t)ctx->n;
        a.R = R;
        a.n_pad = (int32_t)tc_pad(ctx->n);
        a.k = k0;
        a.k_end = k1;
        a.dt = dt;
        a.a0 = a0;
        a.c0 = c0;
        // a launch after an odd number of steps starts from the other buffers
        const bool flip = ((k0 - k_begin) & 1) != 0;
        a.S_a = flip ? S_b : S_a;
        a.S_b = field_only ? nullptr : (flip ? const_cast<float*>(S_a) : S_b);
        a.Y = Y;
        a.sop[0] = sop ? sop[0] : nullptr;
        a.sop[1] = sop ? sop[1] : nullptr;
        a.cur = (cur + (k0 - k_begin)) & 1;
        a.colmajor = steps > 1 ? (int32_t)std::min<int64_t>(tc_column_group(prec, terms), NT) : 0;
        a.bf = ctx->bf.as<float>();
        a.qscale = ctx->qscale8.as<float>();
        a.a_table = a_table;
        a.F_out = k1 == k_end ? F_out : nullptr;
        a.err = err;
        a.alpha = rule.alpha;
        a.plane = (int64_t)R * a.n_pad;
        a.done = nullptr;
        if (steps > 1) {
            // sized by the caller before any stream capture (256 replicas per column block)
            if (ctx->tcdone.bytes < sizeof(uint32_t) * (size_t)NT)
                return fail(VELOXQ_EINVAL, "tensor-core run without its completion counters");
            VQ_CUDA(cudaMemsetAsync(ctx->tcdone.p, 0, sizeof(uint32_t) * (size_t)NT, ctx->stream));
            a.done = ctx->tcdone.as<uint32_t>();
        }
        const int64_t pairs = std::max<int64_t>(1, std::min<int64_t>(tiles * steps, max_pairs));
        cfg.gridDim = dim3((unsigned)(2 * pairs));
        cfg.numAttrs = 2;   // with programmatic dependent launch (the occupancy query above used the cluster only)
        VQ_CUDA(cudaLaunchKernelEx(&cfg, fn, mq, ms[0], ms[1], lo0, lo1, a));
        VQ_LAUNCH_CHECK("tc step");
    }
    return VELOXQ_OK;
}

// The field alone, F = Qoff S, from the operand behind ms (and ms_lo).
int tc_field(veloxq_ctx* ctx, int prec, int32_t R, const CUtensorMap& mq, const CUtensorMap& ms,
             const CUtensorMap* ms_lo, float* F_out, int* err) {
    const CUtensorMap mss[2] = {ms, ms};
    CUtensorMap lo[2];
    if (ms_lo) lo[0] = lo[1] = *ms_lo;
    return tc_run(ctx, prec, R, mq, mss, ms_lo ? lo : nullptr, 0, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 1,
                  0.f, 0.f, 0.f, F_out, err, Rule());
}

}  // namespace vq
