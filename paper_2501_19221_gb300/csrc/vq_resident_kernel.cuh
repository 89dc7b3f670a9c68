// vq_resident_kernel.cuh -- the whole run of a sparse instance in ONE launch
// (kernel template). Each vq_resident_rc*.cu instantiates the variants for
// one replica count per CTA, so the variants compile in parallel.
//
// Replicas are independent (App. B: many replicas evolved in parallel, the
// best kept), so a CTA owns RC replicas and every variable of them: their
// positions s live in shared memory (two buffers, variable-major [n][RC]),
// their momenta y in registers, the CSR rows of Qs in shared memory when
// they fit. A step needs no communication beyond the CTA: field, update,
// walls, readout, exact energy and best-so-far all stay on chip, with one
// __syncthreads per step. Only the final best energies and bit vectors are
// written to global memory.
#pragma once
#include <cuda_fp16.h>

#include <algorithm>

#include "vq_internal.cuh"

namespace vq {

namespace resident {

constexpr int kSmemMax = 232448;   // 227 KB opt-in per CTA

struct ResArgs {
    int32_t n, R, K, k_begin, k_end, readout_every, nwords;
    int32_t ell_d;         // ELL layout: slots per row (even), else 0
    int32_t method;        // veloxq_method
    float alpha;           // PA momentum
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
// in-line position, as in Chimera cells) land on different banks. (Moving
// the 32-byte rows of RC = 8 as whole pairs over 4 positions instead, which
// keeps a row's second chunk at +16 bytes, made the Chimera C16 solve 32%
// slower.)
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
// value as an exact half in the upper 16 bits of one word, with the float
// offset of the neighbour's state row in the lower 16 bits.
//
// ELL (integer instances whose rows are nearly equally long, such as Chimera
// graphs and lattices): slot p of row i is word [p * n + i], so the threads of
// a warp read consecutive words (no bank conflicts, no row pointers); rows
// shorter than the slot count are padded with a zero weight on the row's own
// state, which adds an exact zero to the field and to the energy.
template <bool PACKED> struct Ent;
template <> struct Ent<true> { uint32_t w; };
template <> struct Ent<false> { uint16_t c; };

struct SmemPlan {
    size_t s0, s1, b, rp, col, val, bits, red, best, flag, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline SmemPlan plan_smem(int n, int64_t nnz, int RC, int threads, int nwords, bool csr_smem,
                                              bool packed, int ell_d) {
    SmemPlan p;
    size_t o = 0;
    const size_t rows = (size_t)((n * RC + 31) / 32 * 32);   // whole 128-byte lines (swizzle)
    p.s0 = o; o = align16(o + sizeof(float) * rows);
    p.s1 = o; o = align16(o + sizeof(float) * rows);
    p.b = o; o = align16(o + sizeof(float) * (size_t)n);
    p.rp = o; o = align16(o + (csr_smem && ell_d == 0 ? sizeof(int32_t) * (size_t)(n + 1) : 0));
    p.col = o; o = align16(o + (ell_d > 0 ? 4 * (size_t)ell_d * n : csr_smem ? (packed ? 4 : 2) * (size_t)nnz : 0));
    p.val = o; o = align16(o + (csr_smem && !packed ? sizeof(float) * (size_t)nnz : 0));
    p.bits = o; o = align16(o + sizeof(uint32_t) * (size_t)RC * nwords);
    p.red = o; o = align16(o + sizeof(int64_t) * (size_t)(threads / 32) * RC);
    p.best = o; o = align16(o + sizeof(int64_t) * RC);
    p.flag = o; o = align16(o + sizeof(int32_t) * RC);
    p.total = o;
    return p;
}

// acc[r] += w * sj[r] (two lanes per instruction where RC >= 2; the same
// bits as scalar fmaf). Measured on the Chimera C16 solve: 13.7 ms against
// 14.0 ms for the scalar form.
template <int RC> __device__ __forceinline__ void acc_fma(float (&acc)[RC], float w, const float (&sj)[RC]) {
    if constexpr (RC >= 2) {
#pragma unroll
        for (int r = 0; r < RC; r += 2) vqd::fma2(acc[r], acc[r + 1], w, w, sj[r], sj[r + 1], acc[r], acc[r + 1]);
    } else {
        acc[0] = fmaf(w, sj[0], acc[0]);
    }
}

__device__ __forceinline__ float ent_w(uint32_t e) { return __half2float(__ushort_as_half((unsigned short)(e >> 16))); }

// Parallel Annealing's binarised spins (+-1) as BF16 at the same element
// index as the float layout (a row of RC = 8 is two 8-byte pieces at 2 o and
// 2 (o ^ 4) bytes): half the bytes of the state per neighbour read, and
// +-1 is exact. A BF16 value is the upper half of its FP32 bits.
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }
__device__ __forceinline__ uint32_t sign_bits(float x) { return vqd::pa_sign(x) > 0.0f ? 0x3F80u : 0xBF80u; }
template <int RC> __device__ __forceinline__ void ld_spin_at(const uint16_t* g, int o, float (&v)[RC]) {
    if constexpr (RC >= 4) {
#pragma unroll
        for (int h = 0; h < RC / 4; ++h) {
            const uint2 a = *reinterpret_cast<const uint2*>(g + (h == 0 ? o : (o ^ 4)));
            v[4 * h] = bf_lo(a.x); v[4 * h + 1] = bf_hi(a.x); v[4 * h + 2] = bf_lo(a.y); v[4 * h + 3] = bf_hi(a.y);
        }
    } else if constexpr (RC == 2) {
        const uint32_t a = *reinterpret_cast<const uint32_t*>(g + o);
        v[0] = bf_lo(a); v[1] = bf_hi(a);
    } else {
        v[0] = __uint_as_float((uint32_t)g[o] << 16);
    }
}
template <int RC> __device__ __forceinline__ void ld_spin(const uint16_t* g, int j, float (&v)[RC]) {
    if constexpr (RC >= 4) ld_spin_at<RC>(g, soff<RC>(j, 0), v);
    else ld_spin_at<RC>(g, j * RC, v);
}
template <int RC> __device__ __forceinline__ void st_spin(uint16_t* g, int j, const float (&x)[RC]) {
    if constexpr (RC >= 4) {
#pragma unroll
        for (int h = 0; h < RC / 4; ++h) {
            uint2 a;
            a.x = sign_bits(x[4 * h]) | (sign_bits(x[4 * h + 1]) << 16);
            a.y = sign_bits(x[4 * h + 2]) | (sign_bits(x[4 * h + 3]) << 16);
            *reinterpret_cast<uint2*>(g + soff<RC>(j, h)) = a;
        }
    } else if constexpr (RC == 2) {
        *reinterpret_cast<uint32_t*>(g + 2 * j) = sign_bits(x[0]) | (sign_bits(x[1]) << 16);
    } else {
        g[j] = (uint16_t)sign_bits(x[0]);
    }
}

// METHOD: the integrator (veloxq_method). For PA the first state buffer
// holds the analog spins x, read and written only by their owner thread, and
// the second holds two BF16 buffers of their binarised spins (the field's
// operand), current and next; readouts take x = [spin > 0] = [x > 0]. ELL: 0, rows in
// CSR form; 6, six slots per row (Chimera graphs, cubic lattices), a count
// known here, so the slot loops unroll completely; 1, a.ell_d slots; 32, at
// most 32 slots with one row per thread (RPT = 1): the thread keeps its row's
// coupling words in registers for the whole run, so a step issues the
// neighbours' loads back to back instead of each behind a shared-memory load
// of its coupling word (small dense instances, whose steps are latency-bound).
template <int RC, int RPT, bool CSR_SMEM, bool PACKED, int MAXT, int ELL, int METHOD>
__global__ void __launch_bounds__(MAXT, 1) k_resident(const ResArgs a) {
    constexpr bool SIGN = METHOD == vqd::METHOD_PA;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = a.n;
    const int ELLD = ELL == 6 ? 6 : a.ell_d;   // slots per row (ELL != 0)
    static_assert(ELL != 32 || RPT == 1, "coupling words in registers need one row per thread");
    const int T = blockDim.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int r0 = blockIdx.x * RC;
    const SmemPlan pl = plan_smem(n, CSR_SMEM ? a.rowptr[n] : 0, RC, T, a.nwords, CSR_SMEM, PACKED, ELL ? a.ell_d : 0);
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
    if constexpr (ELL != 0) {
        const int64_t tot = (int64_t)ELLD * n;
        for (int64_t idx = tid; idx < tot; idx += T) {
            const int p = (int)(idx / n), i = (int)(idx - (int64_t)p * n);
            const int64_t q0 = a.rowptr[i];
            uint32_t e = (uint32_t)soff<RC>(i, 0);   // padding: weight +0 on the own row
            if (q0 + p < a.rowptr[i + 1])
                e = (uint32_t)soff<RC>(a.col[q0 + p], 0) |
                    ((uint32_t)__half_as_ushort(__float2half_rn(a.wf[q0 + p])) << 16);
            packs[idx] = e;
        }
    } else if constexpr (CSR_SMEM) {
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
    // PA: the two spin buffers share the second state region
    uint16_t* gc = reinterpret_cast<uint16_t*>(sB);
    uint16_t* gn = gc + (pl.s1 - pl.s0) / sizeof(float);
    if constexpr (SIGN) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int i = tid + q * T;
            if (i < n) {
                float x[RC];
                ld_row<RC>(sA, i, x);
                st_spin<RC>(gc, i, x);
            }
        }
    }
    __syncthreads();

    // ELL == 32: this thread's row of coupling words, held for the whole run
    uint32_t pk[ELL == 32 ? 32 : 1];
    if constexpr (ELL == 32) {
#pragma unroll
        for (int p = 0; p < 32; ++p) pk[p] = (p < ELLD && tid < n) ? packs[(int64_t)p * n + tid] : 0u;
    }
    float* sc = sA;
    float* sn = SIGN ? sA : sB;
    // a neighbour's field operand: its state row, or (PA) its spin row
    auto nb_at = [&](int o, float (&v)[RC]) {
        if constexpr (SIGN) ld_spin_at<RC>(gc, o, v);
        else ld_row_at<RC>(sc, o, v);
    };
    auto nb_row = [&](int j, float (&v)[RC]) {
        if constexpr (SIGN) ld_spin<RC>(gc, j, v);
        else ld_row<RC>(sc, j, v);
    };
    for (int k = a.k_begin; k < a.k_end; ++k) {
        const float a_k = __ldg(a.a_table + k);
        const bool last = (k == a.k_end - 1);
        // field of row i into acc (slot order = CSR order)
        auto row_field = [&](int i, float (&acc)[RC]) {
#pragma unroll
            for (int r = 0; r < RC; ++r) acc[r] = 0.0f;
            if constexpr (ELL == 32) {
                // slot order, as in the other layouts
#pragma unroll
                for (int p = 0; p < 32; ++p)
                    if (p < ELLD) {
                        float sj[RC];
                        nb_at((int)(pk[p] & 0xFFFFu), sj);
                        acc_fma<RC>(acc, ent_w(pk[p]), sj);
                    }
            } else if constexpr (ELL != 0) {
                // two slots per iteration: both neighbours' loads are in flight together
                const uint32_t* e = packs + i;
#pragma unroll
                for (int p = 0; p < ELLD; p += 2, e += 2 * n) {
                    const uint32_t e0 = e[0], e1 = e[n];
                    float s0[RC], s1[RC];
                    nb_at((int)(e0 & 0xFFFFu), s0);
                    nb_at((int)(e1 & 0xFFFFu), s1);
                    acc_fma<RC>(acc, ent_w(e0), s0);
                    acc_fma<RC>(acc, ent_w(e1), s1);
                }
            } else {
                int p0, p1;
                if constexpr (CSR_SMEM) { p0 = rps[i]; p1 = rps[i + 1]; }
                else { p0 = (int)__ldg(a.rowptr + i); p1 = (int)__ldg(a.rowptr + i + 1); }
                for (int p = p0; p < p1; ++p) {
                    float w;
                    float sj[RC];
                    if constexpr (CSR_SMEM && PACKED) {
                        const uint32_t e = packs[p];
                        w = ent_w(e);
                        nb_at((int)(e & 0xFFFFu), sj);
                    } else {
                        int j;
                        if constexpr (CSR_SMEM) { j = cols[p]; w = vals[p]; }
                        else { j = __ldg(a.col + p); w = __ldg(a.wf + p); }
                        nb_row(j, sj);
                    }
                    acc_fma<RC>(acc, w, sj);
                }
            }
        };
        // fields of rows i and i + T together (ELL): four neighbours' loads in flight
        auto pair_field = [&](int i, float (&acc0)[RC], float (&acc1)[RC]) {
#pragma unroll
            for (int r = 0; r < RC; ++r) { acc0[r] = 0.0f; acc1[r] = 0.0f; }
            const uint32_t* e = packs + i;
            const uint32_t* f = packs + i + T;
#pragma unroll
            for (int p = 0; p < ELLD; p += 2, e += 2 * n, f += 2 * n) {
                const uint32_t e0 = e[0], e1 = e[n], f0 = f[0], f1 = f[n];
                float s0[RC], s1[RC], t0[RC], t1[RC];
                nb_at((int)(e0 & 0xFFFFu), s0);
                nb_at((int)(e1 & 0xFFFFu), s1);
                nb_at((int)(f0 & 0xFFFFu), t0);
                nb_at((int)(f1 & 0xFFFFu), t1);
                acc_fma<RC>(acc0, ent_w(e0), s0);
                acc_fma<RC>(acc0, ent_w(e1), s1);
                acc_fma<RC>(acc1, ent_w(f0), t0);
                acc_fma<RC>(acc1, ent_w(f1), t1);
            }
        };
        // update of row i (the q-th of this thread) from its field, into the next buffer
        auto finish = [&](int q, int i, const float (&acc)[RC]) {
            float s[RC];
            ld_row<RC>(sc, i, s);
            const float b = bsh[i];
            if constexpr (METHOD == vqd::METHOD_PA) {
                const float lam = vqd::pa_lambda(a_k, a.a0);
                if constexpr (RC >= 2) {
#pragma unroll
                    for (int r = 0; r < RC; r += 2)
                        vqd::pa_update2(acc[r], acc[r + 1], b, lam, a.dt, a.alpha, a.c0, s[r], s[r + 1], y[q][r],
                                        y[q][r + 1]);
                } else {
                    vqd::pa_update(acc[0], b, lam, a.dt, a.alpha, a.c0, s[0], y[q][0]);
                }
            } else if constexpr (METHOD == vqd::METHOD_ASB) {
                if constexpr (RC >= 2) {
#pragma unroll
                    for (int r = 0; r < RC; r += 2)
                        vqd::asb_update2(acc[r], acc[r + 1], b, a_k, a.dt, a.a0, a.c0, s[r], s[r + 1], y[q][r],
                                         y[q][r + 1]);
                } else {
                    vqd::asb_update(acc[0], b, a_k, a.dt, a.a0, a.c0, s[0], y[q][0]);
                }
            } else if constexpr (RC >= 2) {
                // two-lane update (measured with scalar accumulation: 14.0 ms per Chimera C16 solve
                // against 15.3 ms for the scalar update)
#pragma unroll
                for (int r = 0; r < RC; r += 2)
                    vqd::bsb_update2(acc[r], acc[r + 1], b, a_k, a.dt, a.a0, a.c0, s[r], s[r + 1], y[q][r],
                                     y[q][r + 1]);
            } else {
                vqd::bsb_update(acc[0], b, a_k, a.dt, a.a0, a.c0, s[0], y[q][0]);
            }
            st_row<RC>(sn, i, s);
            if constexpr (SIGN) st_spin<RC>(gn, i, s);
            if (last && a.F_out) {
#pragma unroll
                for (int r = 0; r < RC; ++r)
                    if (r0 + r < a.R) a.F_out[(int64_t)(r0 + r) * n + i] = acc[r];
            }
        };
        constexpr bool PAIRS = ELL != 0 && RPT >= 2;
#pragma unroll
        for (int q = 0; q < RPT; q += PAIRS ? 2 : 1) {
            const int i = tid + q * T;
            if constexpr (PAIRS) {
                if (i + T < n) {
                    float acc0[RC], acc1[RC];
                    pair_field(i, acc0, acc1);
                    finish(q, i, acc0);
                    finish(q + 1, i + T, acc1);
                } else if (i < n) {
                    float acc[RC];
                    row_field(i, acc);
                    finish(q, i, acc);
                }
            } else if (i < n) {
                float acc[RC];
                row_field(i, acc);
                finish(q, i, acc);
            }
        }
        __syncthreads();
        if constexpr (SIGN) {
            uint16_t* t = gc; gc = gn; gn = t;      // x stays in its one buffer
        } else {
            float* tmp = sc; sc = sn; sn = tmp;
        }

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
                nb_row(i, si);
                bool any = false;
#pragma unroll
                for (int r = 0; r < RC; ++r) any |= si[r] > 0.0f;
                if (any) {
                    int64_t row[RC];
#pragma unroll
                    for (int r = 0; r < RC; ++r) row[r] = 0;
                    if constexpr (ELL != 0) {
                        // integer instances only: 2 Qs is exact from the half value
                        const uint32_t* e = packs + i;
#pragma unroll
                        for (int p = 0; p < ELLD; ++p, e += n) {
                            const uint32_t ev = e[0];
                            float sj[RC];
                            nb_at((int)(ev & 0xFFFFu), sj);
                            const int64_t wq = (int64_t)__float2int_rn(2.0f * ent_w(ev));
#pragma unroll
                            for (int r = 0; r < RC; ++r) row[r] += sj[r] > 0.0f ? wq : 0;
                        }
                    } else {
                    int p0, p1;
                    if constexpr (CSR_SMEM) { p0 = rps[i]; p1 = rps[i + 1]; }
                    else { p0 = (int)__ldg(a.rowptr + i); p1 = (int)__ldg(a.rowptr + i + 1); }
                    for (int p = p0; p < p1; ++p) {
                        float w;
                        float sj[RC];
                        if constexpr (CSR_SMEM && PACKED) {
                            const uint32_t e = packs[p];
                            w = ent_w(e);
                            nb_at((int)(e & 0xFFFFu), sj);
                        } else {
                            int j;
                            if constexpr (CSR_SMEM) { j = cols[p]; w = vals[p]; }
                            else { j = __ldg(a.col + p); w = __ldg(a.wf + p); }
                            nb_row(j, sj);
                        }
                        // 2 Qs for integer instances (exact), the fixed-point weight otherwise
                        const int64_t wq = a.wfix ? __ldg(a.wfix + p) : (int64_t)__float2int_rn(2.0f * w);
#pragma unroll
                        for (int r = 0; r < RC; ++r) row[r] += sj[r] > 0.0f ? wq : 0;
                    }
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
template <int RC, int RPT, int METHOD> KFn pick_csr(bool csr_smem, bool packed, int ell_d, int threads) {
    constexpr int MAXT = (RC * RPT <= 8) ? 1024 : 512;
    if constexpr (RC * RPT > 32) {
        return nullptr;   // never planned (the momenta do not fit in registers)
    } else {
        if (!csr_smem) return k_resident<RC, RPT, false, false, MAXT, 0, METHOD>;
        if constexpr (RPT == 1) {
            // the 32 coupling words need the 128-register budget of a 512-thread CTA
            if (ell_d > 0 && ell_d <= 32 && threads <= 512) return k_resident<RC, 1, true, true, 512, 32, METHOD>;
        }
        if (ell_d == 6) return k_resident<RC, RPT, true, true, MAXT, 6, METHOD>;
        if (ell_d > 0) return k_resident<RC, RPT, true, true, MAXT, 1, METHOD>;
        return packed ? k_resident<RC, RPT, true, true, MAXT, 0, METHOD>
                      : k_resident<RC, RPT, true, false, MAXT, 0, METHOD>;
    }
}

// the variants of one replica count per CTA and one integrator
template <int RC, int METHOD> KFn pick_rpt(int rpt, bool csr_smem, bool packed, int ell, int threads) {
    switch (rpt) {
        case 1: return pick_csr<RC, 1, METHOD>(csr_smem, packed, ell, threads);
        case 2: return pick_csr<RC, 2, METHOD>(csr_smem, packed, ell, threads);
        case 4: return pick_csr<RC, 4, METHOD>(csr_smem, packed, ell, threads);
        case 8: return pick_csr<RC, 8, METHOD>(csr_smem, packed, ell, threads);
        default: return pick_csr<RC, 16, METHOD>(csr_smem, packed, ell, threads);
    }
}

}  // namespace resident

// one per replica count per CTA and integrator (vq_resident_*.cu, compiled in parallel)
#define VQ_RESIDENT_PICK(RC, M) \
    resident::KFn resident_pick_rc##RC##_m##M(int rpt, bool csr_smem, bool packed, int ell, int threads)
VQ_RESIDENT_PICK(1, 0); VQ_RESIDENT_PICK(2, 0); VQ_RESIDENT_PICK(4, 0); VQ_RESIDENT_PICK(8, 0);
VQ_RESIDENT_PICK(1, 1); VQ_RESIDENT_PICK(2, 1); VQ_RESIDENT_PICK(4, 1); VQ_RESIDENT_PICK(8, 1);
VQ_RESIDENT_PICK(1, 2); VQ_RESIDENT_PICK(2, 2); VQ_RESIDENT_PICK(4, 2); VQ_RESIDENT_PICK(8, 2);

}  // namespace vq
