// vq_resident.cu -- the whole run of a sparse instance in ONE launch.
//
// Replicas are independent (App. B: many replicas evolved in parallel, the
// best kept), so a CTA owns RC replicas and every variable of them: their
// positions s live in shared memory (two buffers, variable-major [n][RC]),
// their momenta y in registers, the CSR rows of Qs in shared memory when
// they fit. A step needs no communication beyond the CTA: field, update,
// walls, readout, exact energy and best-so-far all stay on chip, with one
// __syncthreads per step. Only the final best energies and bit vectors are
// written to global memory.
#include <cuda_fp16.h>

#include <algorithm>

#include "vq_internal.cuh"

namespace vq {

namespace {

constexpr int kSmemMax = 232448;   // 227 KB opt-in per CTA

struct ResArgs {
    int32_t n, R, K, k_begin, k_end, readout_every, nwords;
    float dt, a0, c0, sigma0;
    uint64_t seed;
    const int64_t* rowptr;
    const int32_t* col;
    const float* wf;
    const int64_t* wfix;   // real instances: round(Qs 2^S); integer: null (2Qs = 2 wf exactly)
    const int64_t* dfix;
    const float* bf;
    const float* a_table;
    const float* S_in;     // [R][n] or null (Philox)
    const float* Y_in;
    float* S_out;          // [R][n] or null
    float* Y_out;
    float* F_out;          // [R][n] field of the last step, or null
    int64_t* best_e;       // [R]
    uint32_t* best_bits;   // [R][nwords]
};

// Shared-memory layout of the positions: variable-major, RC replicas per
// variable. For RC >= 4 the 16-byte chunks of a row are XOR-swizzled across
// the 128-byte line by the line index, so rows 4 or 8 apart (the same
// in-line position, as in Chimera cells) land on different banks.
template <int RC> __device__ __forceinline__ int soff(int j, int h) {
    if constexpr (RC >= 4) {
        const int line = (j * RC) >> 5;
        const int c = ((j * RC) >> 2) & 7;
        return (line << 5) + ((((c + h) ^ line) & 7) << 2);
    } else {
        return j * RC;
    }
}
template <int RC> __device__ __forceinline__ int selem(int j, int r) {
    if constexpr (RC >= 4) return soff<RC>(j, r >> 2) + (r & 3);
    else return j * RC + r;
}
template <int RC> __device__ __forceinline__ void ld_row(const float* s, int j, float (&v)[RC]) {
    if constexpr (RC >= 4) {
#pragma unroll
        for (int h = 0; h < RC / 4; ++h) {
            const float4 a = *reinterpret_cast<const float4*>(s + soff<RC>(j, h));
            v[4 * h] = a.x; v[4 * h + 1] = a.y; v[4 * h + 2] = a.z; v[4 * h + 3] = a.w;
        }
    } else if constexpr (RC == 2) {
        const float2 a = *reinterpret_cast<const float2*>(s + 2 * j);
        v[0] = a.x; v[1] = a.y;
    } else {
        v[0] = s[j];
    }
}
// The same load given the float offset of the row's first chunk (the second
// chunk of an 8-replica row is at offset ^ 4: the chunk pair is XOR-swizzled
// together).
template <int RC> __device__ __forceinline__ void ld_row_at(const float* s, int o, float (&v)[RC]) {
    if constexpr (RC == 8) {
        const float4 a = *reinterpret_cast<const float4*>(s + o);
        const float4 b = *reinterpret_cast<const float4*>(s + (o ^ 4));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else if constexpr (RC == 4) {
        const float4 a = *reinterpret_cast<const float4*>(s + o);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else if constexpr (RC == 2) {
        const float2 a = *reinterpret_cast<const float2*>(s + o);
        v[0] = a.x; v[1] = a.y;
    } else {
        v[0] = s[o];
    }
}
template <int RC> __device__ __forceinline__ void st_row(float* s, int j, const float (&v)[RC]) {
    if constexpr (RC >= 4) {
#pragma unroll
        for (int h = 0; h < RC / 4; ++h)
            *reinterpret_cast<float4*>(s + soff<RC>(j, h)) = make_float4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
    } else if constexpr (RC == 2) {
        *reinterpret_cast<float2*>(s + 2 * j) = make_float2(v[0], v[1]);
    } else {
        s[j] = v[0];
    }
}

// A coupling in shared memory: column (16 bits) and value. PACKED stores the
// value as an exact half in the upper 16 bits of one word.
template <bool PACKED> struct Ent;
template <> struct Ent<true> { uint32_t w; };
template <> struct Ent<false> { uint16_t c; };

struct SmemPlan {
    size_t s0, s1, b, rp, col, val, bits, red, best, flag, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline SmemPlan plan_smem(int n, int64_t nnz, int RC, int threads, int nwords, bool csr_smem,
                                              bool packed) {
    SmemPlan p;
    size_t o = 0;
    const size_t rows = (size_t)((n * RC + 31) / 32 * 32);   // whole 128-byte lines (swizzle)
    p.s0 = o; o = align16(o + sizeof(float) * rows);
    p.s1 = o; o = align16(o + sizeof(float) * rows);
    p.b = o; o = align16(o + sizeof(float) * (size_t)n);
    p.rp = o; o = align16(o + (csr_smem ? sizeof(int32_t) * (size_t)(n + 1) : 0));
    p.col = o; o = align16(o + (csr_smem ? (packed ? 4 : 2) * (size_t)nnz : 0));
    p.val = o; o = align16(o + (csr_smem && !packed ? sizeof(float) * (size_t)nnz : 0));
    p.bits = o; o = align16(o + sizeof(uint32_t) * (size_t)RC * nwords);
    p.red = o; o = align16(o + sizeof(int64_t) * (size_t)(threads / 32) * RC);
    p.best = o; o = align16(o + sizeof(int64_t) * RC);
    p.flag = o; o = align16(o + sizeof(int32_t) * RC);
    p.total = o;
    return p;
}

template <int RC, int RPT, bool CSR_SMEM, bool PACKED, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_resident(const ResArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = a.n;
    const int T = blockDim.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int r0 = blockIdx.x * RC;
    const SmemPlan pl = plan_smem(n, CSR_SMEM ? a.rowptr[n] : 0, RC, T, a.nwords, CSR_SMEM, PACKED);
    float* sA = reinterpret_cast<float*>(smem + pl.s0);
    float* sB = reinterpret_cast<float*>(smem + pl.s1);
    float* bsh = reinterpret_cast<float*>(smem + pl.b);
    int32_t* rps = reinterpret_cast<int32_t*>(smem + pl.rp);
    uint16_t* cols = reinterpret_cast<uint16_t*>(smem + pl.col);
    uint32_t* packs = reinterpret_cast<uint32_t*>(smem + pl.col);
    float* vals = reinterpret_cast<float*>(smem + pl.val);
    uint32_t* bits = reinterpret_cast<uint32_t*>(smem + pl.bits);
    int64_t* red = reinterpret_cast<int64_t*>(smem + pl.red);
    int64_t* best = reinterpret_cast<int64_t*>(smem + pl.best);
    int32_t* flag = reinterpret_cast<int32_t*>(smem + pl.flag);

    // ---- stage constants ----
    for (int i = tid; i < n; i += T) bsh[i] = a.bf[i];
    if constexpr (CSR_SMEM) {
        const int64_t nnz = a.rowptr[n];
        for (int i = tid; i <= n; i += T) rps[i] = (int32_t)a.rowptr[i];
        for (int64_t p = tid; p < nnz; p += T) {
            if constexpr (PACKED) {
                // low half: the float offset of the neighbour's first chunk in the state layout
                packs[p] = (uint32_t)soff<RC>(a.col[p], 0) | ((uint32_t)__half_as_ushort(__float2half_rn(a.wf[p])) << 16);
            } else {
                cols[p] = (uint16_t)a.col[p];
                vals[p] = a.wf[p];
            }
        }
    }
    for (int w = tid; w < RC * a.nwords; w += T) bits[w] = 0u;
    if (tid < RC) best[tid] = INT64_MAX;

    // ---- initial state: s in shared memory, y in registers ----
    float y[RPT][RC];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int i = tid + q * T;
#pragma unroll
        for (int r = 0; r < RC; ++r) {
            float s = 0.0f, yv = 0.0f;
            if (i < n && r0 + r < a.R) {
                if (a.S_in) {
                    s = a.S_in[(int64_t)(r0 + r) * n + i];
                    yv = a.Y_in[(int64_t)(r0 + r) * n + i];
                } else {
                    vqd::init_pair(i, r0 + r, a.seed, a.sigma0, &s, &yv);
                }
            }
            if (i < n) sA[selem<RC>(i, r)] = s;
            y[q][r] = yv;
        }
    }
    __syncthreads();

    float* sc = sA;
    float* sn = sB;
    for (int k = a.k_begin; k < a.k_end; ++k) {
        const float a_k = __ldg(a.a_table + k);
        const bool last = (k == a.k_end - 1);
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int i = tid + q * T;
            if (i < n) {
                float acc[RC];
#pragma unroll
                for (int r = 0; r < RC; ++r) acc[r] = 0.0f;
                int p0, p1;
                if constexpr (CSR_SMEM) { p0 = rps[i]; p1 = rps[i + 1]; }
                else { p0 = (int)__ldg(a.rowptr + i); p1 = (int)__ldg(a.rowptr + i + 1); }
                for (int p = p0; p < p1; ++p) {
                    float w;
                    float sj[RC];
                    if constexpr (CSR_SMEM && PACKED) {
                        const uint32_t e = packs[p];
                        w = __half2float(__ushort_as_half((unsigned short)(e >> 16)));
                        ld_row_at<RC>(sc, (int)(e & 0xFFFFu), sj);
                    } else {
                        int j;
                        if constexpr (CSR_SMEM) { j = cols[p]; w = vals[p]; }
                        else { j = __ldg(a.col + p); w = __ldg(a.wf + p); }
                        ld_row<RC>(sc, j, sj);
                    }
#pragma unroll
                    for (int r = 0; r < RC; ++r) acc[r] = fmaf(w, sj[r], acc[r]);
                }
                float s[RC];
                ld_row<RC>(sc, i, s);
                const float b = bsh[i];
#pragma unroll
                for (int r = 0; r < RC; ++r) vqd::bsb_update(acc[r], b, a_k, a.dt, a.a0, a.c0, s[r], y[q][r]);
                st_row<RC>(sn, i, s);
                if (last && a.F_out) {
#pragma unroll
                    for (int r = 0; r < RC; ++r)
                        if (r0 + r < a.R) a.F_out[(int64_t)(r0 + r) * n + i] = acc[r];
                }
            }
        }
        __syncthreads();
        float* tmp = sc; sc = sn; sn = tmp;

        const bool readout = (a.readout_every >= 0) &&
                             ((k == a.K - 1) || (a.readout_every > 0 && ((k + 1) % a.readout_every) == 0));
        if (!readout) continue;
        // ---- exact energy of x = [s > 0], fixed point (int64 multiples of 2^-S) ----
        int64_t part[RC];
#pragma unroll
        for (int r = 0; r < RC; ++r) part[r] = 0;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int i = tid + q * T;
            if (i < n) {
                float si[RC];
                ld_row<RC>(sc, i, si);
                bool any = false;
#pragma unroll
                for (int r = 0; r < RC; ++r) any |= si[r] > 0.0f;
                if (any) {
                    int64_t row[RC];
#pragma unroll
                    for (int r = 0; r < RC; ++r) row[r] = 0;
                    int p0, p1;
                    if constexpr (CSR_SMEM) { p0 = rps[i]; p1 = rps[i + 1]; }
                    else { p0 = (int)__ldg(a.rowptr + i); p1 = (int)__ldg(a.rowptr + i + 1); }
                    for (int p = p0; p < p1; ++p) {
                        float w;
                        float sj[RC];
                        if constexpr (CSR_SMEM && PACKED) {
                            const uint32_t e = packs[p];
                            w = __half2float(__ushort_as_half((unsigned short)(e >> 16)));
                            ld_row_at<RC>(sc, (int)(e & 0xFFFFu), sj);
                        } else {
                            int j;
                            if constexpr (CSR_SMEM) { j = cols[p]; w = vals[p]; }
                            else { j = __ldg(a.col + p); w = __ldg(a.wf + p); }
                            ld_row<RC>(sc, j, sj);
                        }
                        // 2 Qs for integer instances (exact), the fixed-point weight otherwise
                        const int64_t wq = a.wfix ? __ldg(a.wfix + p) : (int64_t)__float2int_rn(2.0f * w);
#pragma unroll
                        for (int r = 0; r < RC; ++r) row[r] += sj[r] > 0.0f ? wq : 0;
                    }
                    const int64_t d = __ldg(a.dfix + i);
#pragma unroll
                    for (int r = 0; r < RC; ++r) part[r] += si[r] > 0.0f ? d + row[r] : 0;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RC; ++r) {
            int64_t v = part[r];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp * RC + r] = v;
        }
        __syncthreads();
        if (tid < RC) {
            int64_t tot = 0;
            for (int w = 0; w < (T >> 5); ++w) tot += red[w * RC + tid];
            const bool better = tot < best[tid];
            if (better) best[tid] = tot;
            flag[tid] = better ? 1 : 0;
        }
        __syncthreads();
        // save the bits of improved replicas: a warp covers 32 consecutive variables
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int i = tid + q * T;
            const int base = warp * 32 + q * T;
            if (base < n) {
#pragma unroll
                for (int r = 0; r < RC; ++r) {
                    if (!flag[r]) continue;
                    const bool bit = (i < n) && sc[selem<RC>(i, r)] > 0.0f;
                    const uint32_t word = __ballot_sync(0xffffffffu, bit);
                    if (lane == 0) bits[r * a.nwords + (base >> 5)] = word;
                }
            }
        }
        // flags are next written after at least one more __syncthreads
    }
    __syncthreads();

    // ---- write results ----
    if (a.best_e && tid < RC && r0 + tid < a.R) a.best_e[r0 + tid] = best[tid];
    if (a.best_bits)
        for (int w = tid; w < RC * a.nwords; w += T) {
            const int r = w / a.nwords;
            if (r0 + r < a.R) a.best_bits[(int64_t)(r0 + r) * a.nwords + (w - r * a.nwords)] = bits[w];
        }
    if (a.S_out) {
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int i = tid + q * T;
            if (i >= n) continue;
#pragma unroll
            for (int r = 0; r < RC; ++r)
                if (r0 + r < a.R) {
                    a.S_out[(int64_t)(r0 + r) * n + i] = sc[selem<RC>(i, r)];
                    a.Y_out[(int64_t)(r0 + r) * n + i] = y[q][r];
                }
        }
    }
}

using KFn = void (*)(const ResArgs);

// 1024-thread CTAs keep at most 8 momenta per thread in registers (64-register
// cap); 512-thread CTAs up to 32.
template <int RC, int RPT> KFn pick_csr(bool csr_smem, bool packed) {
    constexpr int MAXT = (RC * RPT <= 8) ? 1024 : 512;
    if (!csr_smem) return k_resident<RC, RPT, false, false, MAXT>;
    return packed ? k_resident<RC, RPT, true, true, MAXT> : k_resident<RC, RPT, true, false, MAXT>;
}

template <int RC> KFn pick_rpt(int rpt, bool csr_smem, bool packed) {
    switch (rpt) {
        case 1: return pick_csr<RC, 1>(csr_smem, packed);
        case 2: return pick_csr<RC, 2>(csr_smem, packed);
        case 4: return pick_csr<RC, 4>(csr_smem, packed);
        case 8: return pick_csr<RC, 8>(csr_smem, packed);
        default: return pick_csr<RC, 16>(csr_smem, packed);
    }
}

KFn pick_kernel(int rc, int rpt, bool csr_smem, bool packed) {
    switch (rc) {
        case 1: return pick_rpt<1>(rpt, csr_smem, packed);
        case 2: return pick_rpt<2>(rpt, csr_smem, packed);
        case 4: return pick_rpt<4>(rpt, csr_smem, packed);
        default: return pick_rpt<8>(rpt, csr_smem, packed);
    }
}

struct ResPlan {
    int rc, threads, rpt;
    bool csr_smem, packed;
    size_t smem;
    bool ok;
};

static int pow2_at_least(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Cost model: every SM runs ceil(CTAs / SMs) CTAs one after another or
// interleaved, and a CTA step costs about (3 + RC) instructions per coupling
// (the column and value loads are shared by its RC replicas).
ResPlan make_plan(const veloxq_ctx* ctx, int32_t R) {
    ResPlan best{0, 0, 0, false, false, 0, false};
    if (!ctx->has_csr || ctx->n > 8192 || ctx->n < 1 || ctx->nnz >= (int64_t)1 << 31) return best;
    const int n = (int)ctx->n;
    const int nwords = (int)div_up(n, 32);
    const bool packed0 = ctx->wf_half_exact;
    double best_cost = 1e300;
    for (int rc : {8, 4, 2, 1}) {
        // threads: 1024 if each keeps <= 8 momenta, else 512 with <= 32
        int threads = std::min(1024, (int)div_up(n, 32) * 32);
        int rpt = pow2_at_least((int)div_up(n, threads));
        if (rc * rpt > 8) {
            threads = std::min(512, (int)div_up(n, 32) * 32);
            rpt = pow2_at_least((int)div_up(n, threads));
            if (rc * rpt > 32 || rpt > 16) continue;
        }
        // packed words hold the row's float offset in 16 bits
        const bool packed = packed0 && (int64_t)div_up((int64_t)n * rc, 32) * 32 <= 65536;
        for (int cs = 1; cs >= 0; --cs) {
            const bool csr_smem = cs == 1 && ctx->n <= 65535;
            if (cs == 1 && !csr_smem) continue;
            const SmemPlan p = plan_smem(n, csr_smem ? ctx->nnz : 0, rc, threads, nwords, csr_smem, csr_smem && packed);
            if (p.total > (size_t)kSmemMax) continue;
            const int64_t ctas = div_up(R, rc);
            const double cost = (double)div_up(ctas, 152) * (3.0 + rc) * (csr_smem ? 1.0 : 1.3);
            if (cost < best_cost - 1e-9) {
                best_cost = cost;
                best = ResPlan{rc, threads, rpt, csr_smem, csr_smem && packed, p.total, true};
            }
            break;   // the CSR-in-shared-memory variant fits: prefer it for this rc
        }
    }
    return best;
}

}  // namespace

bool resident_fits(const veloxq_ctx* ctx, int32_t R, int* rc, int* threads, size_t* smem) {
    const ResPlan p = make_plan(ctx, R);
    if (rc) *rc = p.rc;
    if (threads) *threads = p.threads;
    if (smem) *smem = p.smem;
    return p.ok;
}

int resident_run(veloxq_ctx* ctx, int32_t R, const RunParams& rp, uint64_t seed, int k_begin, int k_end,
                 const float* S_in, const float* Y_in, float* S_out, float* Y_out, float* F_out, int64_t* best_e,
                 uint32_t* best_bits) {
    const ResPlan p = make_plan(ctx, R);
    if (!p.ok) return fail(VELOXQ_EUNSUPPORTED, "instance does not fit the resident kernel (n <= 8192 sparse, shared memory)");
    ResArgs a;
    a.n = (int32_t)ctx->n;
    a.R = R;
    a.K = rp.K;
    a.k_begin = k_begin;
    a.k_end = k_end;
    a.readout_every = best_e ? rp.readout_every : -1;
    a.nwords = (int32_t)div_up(ctx->n, 32);
    a.dt = rp.dt;
    a.a0 = rp.a0;
    a.c0 = rp.c0;
    a.sigma0 = rp.sigma0;
    a.seed = seed;
    a.rowptr = ctx->rowptr.as<int64_t>();
    a.col = ctx->col.as<int32_t>();
    a.wf = ctx->wf.as<float>();
    a.wfix = ctx->integer ? nullptr : ctx->wfix.as<int64_t>();
    a.dfix = ctx->dfix.as<int64_t>();
    a.bf = ctx->bf.as<float>();
    a.a_table = ctx->a_table.as<float>();
    a.S_in = S_in;
    a.Y_in = Y_in;
    a.S_out = S_out;
    a.Y_out = Y_out;
    a.F_out = F_out;
    a.best_e = best_e;
    a.best_bits = best_bits;
    KFn fn = pick_kernel(p.rc, p.rpt, p.csr_smem, p.packed);
    VQ_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    fn<<<(unsigned)div_up(R, p.rc), p.threads, p.smem, ctx->stream>>>(a);
    VQ_LAUNCH_CHECK("resident kernel");
    return VELOXQ_OK;
}

}  // namespace vq
