// vq_internal.cuh -- internal declarations of libveloxq (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/veloxq.h"

// ---------------------------------------------------------------------------
// error plumbing: every entry point returns a status, the message is
// thread-local.
// ---------------------------------------------------------------------------
namespace vq {

void set_error(const std::string& msg);
int fail(int status, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define VQ_CUDA(call)                                               \
    do {                                                            \
        cudaError_t _e = (call);                                    \
        if (_e != cudaSuccess) return ::vq::cuda_fail(_e, #call);   \
    } while (0)

#define VQ_TRY(call)                    \
    do {                                \
        int _s = (call);                \
        if (_s != VELOXQ_OK) return _s; \
    } while (0)

#define VQ_LAUNCH_CHECK(what)                                           \
    do {                                                                \
        cudaError_t _e = cudaGetLastError();                            \
        if (_e != cudaSuccess) return ::vq::cuda_fail(_e, what);        \
    } while (0)

// Device buffer owned by a context (or by one call, for temporaries). Its
// memory comes from a per-device cache of released blocks when one of a
// fitting size is there, else from cudaMalloc; release() waits for the device
// like cudaFree and returns the block to that cache (vq_api.cu).
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    int dev = -1;               // device the block belongs to
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release();
    // grow to at least `b` bytes (contents not kept)
    int ensure(size_t b);
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

// Row layout of a state block in device memory.
enum Layout { LAYOUT_RN = 0 /* [R][n], replica-major */, LAYOUT_NR = 1 /* [n][R] */ };

// Resolved schedule for one run.
struct RunParams {
    float dt, a0, c0, sigma0;
    float kappa;
    bool c0_given;
    int32_t K;
    int32_t readout_every;
    veloxq_prec prec;
    veloxq_path path;
    int method;                 // veloxq_method
    float alpha;                // PA momentum
    std::vector<double> knots;  // at least 1
};

}  // namespace vq

// ---------------------------------------------------------------------------
// the context
// ---------------------------------------------------------------------------
struct veloxq_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t n = 0;
    bool dense = false;
    bool has_csr = false;         // sparse rows of Qoff present (sparse contexts, small dense ones)
    bool integer = false;
    double K0 = 0.0;
    double rho = 0.0;
    double ising_offset = 0.0;
    int energy_shift = 0;         // fixed-point exponent S: energies are int64 multiples of 2^-S

    // ---- sparse: off-diagonal part of Qs in CSR ----
    int64_t nnz = 0;
    vq::DevBuf rowptr;            // int64 [n+1]
    vq::DevBuf col;               // int32 [nnz]
    vq::DevBuf wf;                // float [nnz]   Qs_ij (field operand)
    vq::DevBuf w8;                // int8  [nnz]   2 Qs_ij when integer and |2Qs| <= 127
    vq::DevBuf wfix;              // int64 [nnz]   round(Qs_ij 2^S) (energy), when w8 is absent
    int max_row = 0;              // longest row of the field structure
    int uniform_deg = -1;         // every row holds this many couplings (-1: rows differ)
    bool wf_half_exact = false;   // every Qs_ij is an exact half (integer |2 Qs| <= 2047)

    // ---- dense ----
    veloxq_vtype qx_type = VELOXQ_F32;
    vq::DevBuf qx;                // [n][n] Q as given (input type; diagonal unused)
    vq::DevBuf qoff32;            // float [n][n] Qoff
    vq::DevBuf qoff16;            // bf16  [n][n] Qoff (tensor-core operand)
    vq::DevBuf qoff8;             // e4m3  [n][n] Qoff / scale_i
    vq::DevBuf qscale8;           // float [n] per-row FP8 scales
    vq::DevBuf qtile;             // pre-tiled swizzled BF16 Qoff for the batched kernel
    size_t qtile_bytes = 0;
    int qtile_fp8 = 0;            // 1: qtile holds the E4M3 form (row scales in qscale8)
    int64_t sop_tag = 0;          // layout the operand buffers sop_a/sop_b last held (0: the single-solve one)
    int32_t batch_R = 0;          // replicas of the state left by the last batched run (0: none)
    // exact readout energies on the tensor cores (vq_energy_tc.cu)
    int eplanes = 0;              // digit planes of round(Q 2^S): 0 not built yet, -1 not used
    vq::DevBuf eplane;            // bf16 [eplanes][n][n_pad] balanced base-256 digits
    vq::DevBuf exop;              // bf16 [R][n_pad] x = [S > 0] (operand)
    vq::DevBuf efield;            // float [R][n] one plane's integer row sums

    // ---- common ----
    vq::DevBuf bf;                // float  [n] b = Qs 1 + c
    vq::DevBuf dfix;              // int64  [n] round((Q_ii + c_i) 2^S)

    // ---- scratch reused across calls ----
    vq::DevBuf s_a, s_b, y, f, ework, best_e, best_bits, flags, a_table, xout, misc;
    vq::DevBuf sop_a, sop_b;      // tensor-core operand copies of S (ping-pong)
    vq::DevBuf dpart;             // float [ksplit][R][n] split-k partial fields of the FP32 dense step
    vq::DevBuf errw;              // device error word of bounded waits
    vq::DevBuf tcdone;            // uint32 [replica column blocks] completion counters of a tensor-core run
    int stream_unroll = 0;        // gather variant of the streaming kernels: 1, 4, or 6 (rows of exactly
                                  // 6 couplings); 0: not tuned yet
    int32_t stream_tuned_R = -1;  // replica count the variant was tuned for
    int32_t stream_cvec = 0;      // replica vectors per chunk of the streaming step's thread order (0: all)
};

namespace vq {

// sizes and helpers
__host__ __device__ inline int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }
int device_sms(int device);   // multiprocessors of a device (queried once per device)

// ingest (vq_ingest.cu)
int ingest_dense(veloxq_ctx* ctx, veloxq_vtype vt, const void* Qh, const double* ch, bool ising);
int ingest_csr(veloxq_ctx* ctx, const int64_t* rowptr, const int32_t* col, veloxq_vtype vt,
               const void* val, const double* ch, bool ising);
int power_iteration(veloxq_ctx* ctx, int iters, double* rho);

// state init, readout, best, argmin (vq_common.cu)
int launch_init_state(veloxq_ctx* ctx, int32_t R, uint64_t seed, float sigma0, Layout layout,
                      float* S, float* Y);
int launch_transpose(cudaStream_t st, const float* in, float* out, int64_t rows, int64_t cols);
int launch_best_update(veloxq_ctx* ctx, int32_t R, int nparts, const int64_t* parts, int64_t* best,
                       uint8_t* improved);
int launch_best_bits(veloxq_ctx* ctx, int32_t R, Layout layout, const float* S, const uint8_t* improved,
                     uint32_t* bits);
int launch_argmin_unpack(veloxq_ctx* ctx, int32_t R, const int64_t* best, const uint32_t* bits,
                         int64_t* misc, uint8_t* x);

// The integrator of a step (veloxq_method) and PA's momentum.
struct Rule {
    int method = 0;
    float alpha = 0.f;
};
inline Rule rule_of(const RunParams& p) { return Rule{p.method, p.alpha}; }

// sparse streaming kernels (vq_stream.cu)
int stream_step(veloxq_ctx* ctx, int32_t R, const float* S_cur, float* S_nxt, float* Y,
                const float* a_table, int k, float dt, float a0, float c0, float* F_out, const Rule& rule = Rule());
int stream_energy(veloxq_ctx* ctx, int32_t R, const float* S, int64_t* parts, int* nparts);
int stream_field(veloxq_ctx* ctx, int32_t R, const float* S, float* F);
int stream_step_y(veloxq_ctx* ctx, int32_t R, const float* S_cur, float* S_nxt, const float* Y_in, float* Y_out,
                  const float* a_table, int k, float dt, float a0, float c0, float* F_out,
                  const Rule& rule = Rule());
int vec_width(int32_t R);
int stream_autotune(veloxq_ctx* ctx, int32_t R, float* S_a, float* S_b, float* Y);

// sparse resident kernel (vq_resident.cu)
bool resident_fits(const veloxq_ctx* ctx, int32_t R, int* rc, int* threads, size_t* smem);
// the resident plan for R replicas keeps the couplings in shared memory
bool resident_on_chip(const veloxq_ctx* ctx, int32_t R);
int resident_run(veloxq_ctx* ctx, int32_t R, const RunParams& p, uint64_t seed, int k_begin, int k_end,
                 const float* S_in, const float* Y_in, float* S_out, float* Y_out, float* F_out,
                 int64_t* best_e, uint32_t* best_bits);

// dense kernels (vq_dense.cu)
int dense_step(veloxq_ctx* ctx, int32_t R, const float* S_cur, float* S_nxt, float* Y,
               const float* a_table, int k, float dt, float a0, float c0, float* F_out, const Rule& rule = Rule());
int dense_field(veloxq_ctx* ctx, int32_t R, const float* S, float* F);
int dense_prepare(veloxq_ctx* ctx, int32_t R);   // workspace of the split-k FP32 step (before capture)
int dense_energy(veloxq_ctx* ctx, int32_t R, const float* S, int64_t* parts, int* nparts, bool allow_tc);
int dense_energy_x(veloxq_ctx* ctx, int64_t B, const uint8_t* X, int64_t* parts, int* nparts, bool allow_tc);
int sparse_energy_x(veloxq_ctx* ctx, int64_t B, const uint8_t* X, int64_t* parts, int* nparts);

// persistent batched kernel (vq_batch.cu)
bool batch_supported(veloxq_ctx* const* ctxs, int32_t count, int32_t R, const RunParams& p);
bool batch_stages_fit(int prec, int method, int stages, int32_t R);   // the form fits shared memory
// The captured device part of a batched solve, reused while its key (every
// pointer, size and parameter its nodes bake in) is unchanged.
struct BatchGraph {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;   // around the persistent kernel
    ~BatchGraph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};
// stages: pipeline depth (4 or 6); split: replica groups per instance, each a
// work item of R / split replicas (a multiple of 16); graph (or null): run the
// device part as a captured graph kept there
int batch_run(veloxq_ctx* const* ctxs, int32_t count, int32_t R, const RunParams& p, uint64_t seed, cudaStream_t st,
              int stages, int split, DevBuf& work, int64_t* d_best_all, int* d_err, float* ms_main,
              int64_t* launches = nullptr, BatchGraph* graph = nullptr);

// adjoint of the step (vq_adjoint.cu); the timing covers the whole gradient
// and, separately, the reverse-step kernels (k_adj_a, k_adj_b, k_adj_reduce)
struct AdjTiming {
    float ms_total = 0.f, ms_reverse = 0.f;
    int64_t launches = 0, reverse_launches = 0;
};
int adjoint_run(veloxq_ctx* ctx, int32_t R, const RunParams& p, const std::vector<float>& a_host, uint64_t seed,
                int32_t C, double* loss, double* d_dt, double* d_c0, double* d_knots, int n_knots, AdjTiming* tm);

// dense tensor-core kernels (vq_tc.cu)
int64_t tc_pad(int64_t n);
int tc_terms(int prec, int method);   // E4M3 terms of the S operand (2 for FP8 unless the operand is exact)
int tc_prepare_q(veloxq_ctx* ctx, int prec);
int tc_maps(veloxq_ctx* ctx, int prec, int terms, int32_t R, void* sop0, void* sop1, CUtensorMap* mq,
            CUtensorMap* ms0, CUtensorMap* ms1, CUtensorMap* ms0_lo, CUtensorMap* ms1_lo);
int tc_quant_s(veloxq_ctx* ctx, int prec, int32_t R, const float* S, void* sop, const Rule& rule = Rule());
size_t tc_sop_bytes(veloxq_ctx* ctx, int prec, int terms, int32_t R);
int tc_wait_selftest(long long budget, int* code_out);   // the bounded wait run out on purpose
// Steps k_begin .. k_end - 1 in one launch (tiles of consecutive steps
// overlap, each waiting only for the column block of the state it reads).
// ms, ms_lo: maps of the two operand buffers sop[0..1] (their lo planes with
// two FP8 terms, else NULL); the first step reads the operand in sop[cur] and
// the state in S_a, and the steps alternate between the two buffers of each
// (after an odd number of steps the state is in S_b and the operand in
// sop[cur ^ 1]). F_out (or NULL): the field of the last step.
int tc_run(veloxq_ctx* ctx, int prec, int32_t R, const CUtensorMap& mq, const CUtensorMap* ms,
           const CUtensorMap* ms_lo, int cur, const float* S_a, float* S_b, float* Y, void* const* sop,
           const float* a_table, int k_begin, int k_end, float dt, float a0, float c0, float* F_out, int* err,
           const Rule& rule = Rule());
// The field alone, F = Qoff S, of the operand behind ms (and ms_lo).
int tc_field(veloxq_ctx* ctx, int prec, int32_t R, const CUtensorMap& mq, const CUtensorMap& ms,
             const CUtensorMap* ms_lo, float* F_out, int* err);
int tc_operand_map(CUtensorMap* m, void* base, int prec, int64_t rows, int64_t n_pad, bool a_operand);
int launch_sum_parts(veloxq_ctx* ctx, int64_t B, int nparts, const int64_t* parts, double* E, int64_t* E_int);

// exact readout energies of a dense instance on the tensor cores (vq_energy_tc.cu)
int tc_energy_prepare(veloxq_ctx* ctx, int64_t R);   // digit planes and workspaces (before capture)
bool tc_energy_ready(const veloxq_ctx* ctx, int64_t R);
int tc_energy(veloxq_ctx* ctx, int64_t R, const float* S, const uint8_t* X, int64_t* parts, int* nparts);

}  // namespace vq

// ---------------------------------------------------------------------------
// device helpers shared by the kernels
// ---------------------------------------------------------------------------
namespace vqd {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
        const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// s0, y0 of variable i, replica r: sigma0 (2u - 1), u = (w >> 8) 2^-24.
__device__ __forceinline__ void init_pair(int64_t i, int32_t r, uint64_t seed, float sigma0, float* s, float* y) {
    uint32_t w[4];
    philox4x32_10((uint32_t)i, (uint32_t)((uint64_t)i >> 32), (uint32_t)r, 0u, (uint32_t)seed,
                  (uint32_t)(seed >> 32), w);
    const float us = __uint2float_rn(w[0] >> 8) * 5.9604644775390625e-8f;
    const float uy = __uint2float_rn(w[1] >> 8) * 5.9604644775390625e-8f;
    *s = __fmul_rn(sigma0, __fsub_rn(__fmul_rn(2.0f, us), 1.0f));
    *y = __fmul_rn(sigma0, __fsub_rn(__fmul_rn(2.0f, uy), 1.0f));
}

// The pieces of one ballistic-SB update before the wall: phi, the drive,
// y-hat and s-hat. Rounded operation by operation (no contraction) so that
// every kernel, the adjoint included, sees the same values.
struct BsbPre {
    float phi, drive, yh, sh;
};
// With t = F + b: drive = -(c0/2) t - (a0 - a_k) s as one fused multiply-add,
// yh = y + dt drive and sh = s + (dt a0) yh likewise (explicit fmaf, the same
// in every kernel).
__device__ __forceinline__ BsbPre bsb_pre(float F, float b, float a_k, float dt, float a0, float c0, float s, float y) {
    BsbPre o;
    const float t = __fadd_rn(F, b);
    o.phi = __fmul_rn(-0.5f, t);
    const float nak = -__fsub_rn(a0, a_k);
    o.drive = fmaf(__fmul_rn(-0.5f, c0), t, __fmul_rn(nak, s));
    o.yh = fmaf(dt, o.drive, y);
    o.sh = fmaf(__fmul_rn(dt, a0), o.yh, s);
    return o;
}

// Two-lane FP32 arithmetic (the packed .f32x2 forms of sm_100 and later):
// each lane is rounded exactly as the scalar instruction rounds it, so the
// results equal the scalar forms bit for bit, at half the issued instructions.
__device__ __forceinline__ void fma2(float& d0, float& d1, float a0, float a1, float b0, float b1, float c0,
                                     float c1) {
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1), "f"(c0), "f"(c1));
}
__device__ __forceinline__ void add2(float& d0, float& d1, float a0, float a1, float b0, float b1) {
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}
__device__ __forceinline__ void mul2(float& d0, float& d1, float a0, float a1, float b0, float b1) {
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// One ballistic-SB update of a single (variable, replica) given its field F:
// y <- y + dt(-(a0 - a_k) s + c0 phi), s <- s + dt a0 y, wall at |s| > 1.
__device__ __forceinline__ void bsb_update(float F, float b, float a_k, float dt, float a0, float c0,
                                           float& s, float& y) {
    const BsbPre o = bsb_pre(F, b, a_k, dt, a0, c0, s, y);
    if (fabsf(o.sh) > 1.0f) {
        s = copysignf(1.0f, o.sh);
        y = 0.0f;
    } else {
        s = o.sh;
        y = o.yh;
    }
}

// The same update for two replicas of one variable (b shared), in the
// two-lane forms: the same operations in the same order as bsb_pre, hence
// the same bits as two calls of bsb_update.
__device__ __forceinline__ void bsb_update2(float F0, float F1, float b, float a_k, float dt, float a0, float c0,
                                            float& s0, float& s1, float& y0, float& y1) {
    float t0, t1, m0, m1, d0, d1, yh0, yh1, sh0, sh1;
    add2(t0, t1, F0, F1, b, b);
    const float nak = -__fsub_rn(a0, a_k);
    mul2(m0, m1, nak, nak, s0, s1);
    const float hc = __fmul_rn(-0.5f, c0);
    fma2(d0, d1, hc, hc, t0, t1, m0, m1);
    fma2(yh0, yh1, dt, dt, d0, d1, y0, y1);
    const float da = __fmul_rn(dt, a0);
    fma2(sh0, sh1, da, da, yh0, yh1, s0, s1);
    if (fabsf(sh0) > 1.0f) { s0 = copysignf(1.0f, sh0); y0 = 0.0f; } else { s0 = sh0; y0 = yh0; }
    if (fabsf(sh1) > 1.0f) { s1 = copysignf(1.0f, sh1); y1 = 0.0f; } else { s1 = sh1; y1 = yh1; }
}

// ---- the other integrators (veloxq_method): adiabatic SB as printed and
// Parallel Annealing; every kernel applies the same operation order ----
enum { METHOD_BSB = 0, METHOD_ASB = 1, METHOD_PA = 2 };

// Field operand of the state: s itself, or PA's binarised spin (+1 where
// s > 0, -1 elsewhere: the readout's rule).
__device__ __forceinline__ float pa_sign(float s) { return s > 0.0f ? 1.0f : -1.0f; }
__device__ __forceinline__ float field_operand(int method, float s) { return method == METHOD_PA ? pa_sign(s) : s; }

// lambda_k = (a0 - a_k)/a0 of Parallel Annealing
__device__ __forceinline__ float pa_lambda(float a_k, float a0) { return __fdiv_rn(__fsub_rn(a0, a_k), a0); }

// y <- y + dt(-(s^2 + a0 - a_k) s + c0 phi), s <- s + dt a0 y (no walls)
__device__ __forceinline__ void asb_update(float F, float b, float a_k, float dt, float a0, float c0, float& s,
                                           float& y) {
    const float t = __fadd_rn(F, b);
    const float coef = __fadd_rn(__fmul_rn(s, s), __fsub_rn(a0, a_k));
    const float drive = fmaf(__fmul_rn(-0.5f, c0), t, -__fmul_rn(coef, s));
    const float yh = fmaf(dt, drive, y);
    s = fmaf(__fmul_rn(dt, a0), yh, s);
    y = yh;
}

// g = lambda x + c0 (F + b)/2, m <- alpha m - dt g, x <- clip(x + m, -1, 1)
__device__ __forceinline__ void pa_update(float F, float b, float lam, float dt, float alpha, float c0, float& x,
                                          float& m) {
    const float t = __fadd_rn(F, b);
    const float g = fmaf(lam, x, __fmul_rn(__fmul_rn(0.5f, c0), t));
    m = fmaf(alpha, m, -__fmul_rn(dt, g));
    x = fminf(fmaxf(__fadd_rn(x, m), -1.0f), 1.0f);
}

// The same two updates for two replicas of one variable, in the two-lane
// forms: the same operations in the same order, hence the same bits.
__device__ __forceinline__ void asb_update2(float F0, float F1, float b, float a_k, float dt, float a0, float c0,
                                            float& s0, float& s1, float& y0, float& y1) {
    float t0, t1, q0, q1, c0v, c1v, m0, m1, d0, d1, yh0, yh1, sn0, sn1;
    add2(t0, t1, F0, F1, b, b);
    mul2(q0, q1, s0, s1, s0, s1);
    const float am = __fsub_rn(a0, a_k);
    add2(c0v, c1v, q0, q1, am, am);
    mul2(m0, m1, c0v, c1v, s0, s1);
    const float hc = __fmul_rn(-0.5f, c0);
    fma2(d0, d1, hc, hc, t0, t1, -m0, -m1);
    fma2(yh0, yh1, dt, dt, d0, d1, y0, y1);
    const float da = __fmul_rn(dt, a0);
    fma2(sn0, sn1, da, da, yh0, yh1, s0, s1);
    s0 = sn0; s1 = sn1; y0 = yh0; y1 = yh1;
}
__device__ __forceinline__ void pa_update2(float F0, float F1, float b, float lam, float dt, float alpha, float c0,
                                           float& x0, float& x1, float& m0, float& m1) {
    float t0, t1, h0, h1, g0, g1, e0, e1, n0, n1, u0, u1;
    add2(t0, t1, F0, F1, b, b);
    const float hc = __fmul_rn(0.5f, c0);
    mul2(h0, h1, hc, hc, t0, t1);
    fma2(g0, g1, lam, lam, x0, x1, h0, h1);
    mul2(e0, e1, dt, dt, g0, g1);
    fma2(n0, n1, alpha, alpha, m0, m1, -e0, -e1);
    add2(u0, u1, x0, x1, n0, n1);
    m0 = n0; m1 = n1;
    x0 = fminf(fmaxf(u0, -1.0f), 1.0f);
    x1 = fminf(fmaxf(u1, -1.0f), 1.0f);
}

// One update of the given method; lam is pa_lambda(a_k, a0) (PA only).
__device__ __forceinline__ void step_update(int method, float F, float b, float a_k, float lam, float dt, float a0,
                                            float c0, float alpha, float& s, float& y) {
    if (method == METHOD_PA) pa_update(F, b, lam, dt, alpha, c0, s, y);
    else if (method == METHOD_ASB) asb_update(F, b, a_k, dt, a0, c0, s, y);
    else bsb_update(F, b, a_k, dt, a0, c0, s, y);
}

// Vector loads/stores of V consecutive replicas.
template <int V> __device__ __forceinline__ void vload(const float* p, float (&v)[V]) {
    if constexpr (V == 4) { const float4 t = __ldg(reinterpret_cast<const float4*>(p)); v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
    else if constexpr (V == 2) { const float2 t = __ldg(reinterpret_cast<const float2*>(p)); v[0] = t.x; v[1] = t.y; }
    else { v[0] = __ldg(p); }
}
template <int V> __device__ __forceinline__ void vload_plain(const float* p, float (&v)[V]) {
    if constexpr (V == 4) { const float4 t = *reinterpret_cast<const float4*>(p); v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
    else if constexpr (V == 2) { const float2 t = *reinterpret_cast<const float2*>(p); v[0] = t.x; v[1] = t.y; }
    else { v[0] = *p; }
}
template <int V> __device__ __forceinline__ void vstore(float* p, const float (&v)[V]) {
    if constexpr (V == 4) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else if constexpr (V == 2) *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    else *p = v[0];
}
// Streaming forms (evict-first in the caches) for data a step touches once,
// so that the state the neighbours gather keeps its place in L2.
template <int V> __device__ __forceinline__ void vload_stream(const float* p, float (&v)[V]) {
    if constexpr (V == 4) { const float4 t = __ldcs(reinterpret_cast<const float4*>(p)); v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
    else if constexpr (V == 2) { const float2 t = __ldcs(reinterpret_cast<const float2*>(p)); v[0] = t.x; v[1] = t.y; }
    else { v[0] = __ldcs(p); }
}
template <int V> __device__ __forceinline__ void vstore_stream(float* p, const float (&v)[V]) {
    if constexpr (V == 4) __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
    else if constexpr (V == 2) __stcs(reinterpret_cast<float2*>(p), make_float2(v[0], v[1]));
    else __stcs(p, v[0]);
}

__device__ __forceinline__ float wval(float w) { return w; }
__device__ __forceinline__ float wval(int8_t w) { return (float)w; }

// acc_l = sum over the CSR row of i of w_p X[col_p][off + l] (variable-major
// [n][R] block), accumulated in CSR order with fmaf. UNROLL = 4 takes four
// couplings per round so that their gathers are in flight together (a slot
// past the row end reads row i itself with weight 0 and adds an exact 0);
// UNROLL = 1 is the plain loop. Both give the same sums.
// acc = sum over row i of w_ij o(X_j) for V replicas, o the identity, (SIGN)
// PA's binarised spin or (SCALE) the product xs X_j, each rounded before it
// enters the sum.
template <int V> __device__ __forceinline__ void sign_vec(float (&v)[V]) {
#pragma unroll
    for (int l = 0; l < V; ++l) v[l] = pa_sign(v[l]);
}
template <int V> __device__ __forceinline__ void scale_vec(float (&v)[V], float xs) {
#pragma unroll
    for (int l = 0; l < V; ++l) v[l] = xs * v[l];
}
template <int V, typename WT, int UNROLL, bool SIGN = false, bool SCALE = false>
__device__ __forceinline__ void csr_row_dot(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                            const WT* __restrict__ w, const float* X, int32_t R, int64_t off,
                                            int64_t i, float (&acc)[V], int udeg = -1, float xs = 1.0f) {
#pragma unroll
    for (int l = 0; l < V; ++l) acc[l] = 0.0f;
    if constexpr (UNROLL == 6) {
        // every row holds exactly 6 couplings (udeg == 6, e.g. cubic
        // lattices): all six columns, then all six neighbour vectors are in
        // flight at once; the sum is taken in CSR order as in the loops below
        const int64_t p0 = i * 6;
        int32_t j[6];
        float wv[6];
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            j[u] = __ldg(col + p0 + u);
            wv[u] = wval(__ldg(w + p0 + u));
        }
        float sj[6][V];
#pragma unroll
        for (int u = 0; u < 6; ++u) vload<V>(X + (int64_t)j[u] * R + off, sj[u]);
        if constexpr (SIGN) {
#pragma unroll
            for (int u = 0; u < 6; ++u) sign_vec<V>(sj[u]);
        }
        if constexpr (SCALE) {
#pragma unroll
            for (int u = 0; u < 6; ++u) scale_vec<V>(sj[u], xs);
        }
#pragma unroll
        for (int u = 0; u < 6; ++u)
#pragma unroll
            for (int l = 0; l < V; ++l) acc[l] = fmaf(wv[u], sj[u][l], acc[l]);
        return;
    }
    // rows of a regular graph start at i * degree: no row pointer is read
    const int64_t p0 = udeg >= 0 ? i * udeg : __ldg(rp + i);
    const int64_t p1 = udeg >= 0 ? p0 + udeg : __ldg(rp + i + 1);
    if constexpr (UNROLL == 1) {
        for (int64_t p = p0; p < p1; ++p) {
            const int64_t j = __ldg(col + p);
            const float wv = wval(__ldg(w + p));
            float sj[V];
            vload<V>(X + j * R + off, sj);
            if constexpr (SIGN) sign_vec<V>(sj);
            if constexpr (SCALE) scale_vec<V>(sj, xs);
#pragma unroll
            for (int l = 0; l < V; ++l) acc[l] = fmaf(wv, sj[l], acc[l]);
        }
    } else {
    for (int64_t p = p0; p < p1; p += 4) {
        int64_t j[4];
        float wv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool on = p + u < p1;
            j[u] = on ? (int64_t)__ldg(col + p + u) : i;
            wv[u] = on ? wval(__ldg(w + p + u)) : 0.0f;
        }
        float sj[4][V];
#pragma unroll
        for (int u = 0; u < 4; ++u) vload<V>(X + j[u] * R + off, sj[u]);
        if constexpr (SIGN) {
#pragma unroll
            for (int u = 0; u < 4; ++u) sign_vec<V>(sj[u]);
        }
        if constexpr (SCALE) {
#pragma unroll
            for (int u = 0; u < 4; ++u) scale_vec<V>(sj[u], xs);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int l = 0; l < V; ++l) acc[l] = fmaf(wv[u], sj[u][l], acc[l]);
    }
    }
}

// Row i and replica vector v of the linear thread index t < n * nvec over n
// rows of nvec vectors; 32-bit divisions when every index fits (a 64-bit
// division costs several times as many instructions).
__device__ __forceinline__ void split_index(int64_t t, int64_t n, int32_t nvec, int64_t& i, int32_t& v) {
    if (nvec == 1) {
        i = t;
        v = 0;
    } else if (n * nvec < (int64_t(1) << 32)) {
        const uint32_t tt = (uint32_t)t, r = tt / (uint32_t)nvec;
        i = r;
        v = (int32_t)(tt - r * (uint32_t)nvec);
    } else {
        i = t / nvec;
        v = (int32_t)(t - i * nvec);
    }
}

// Fixed-point form of a coupling: round(q 2^shift) as int64 (energies).
template <typename QT> __device__ __forceinline__ int64_t qfix(QT q, int shift);
template <> __device__ __forceinline__ int64_t qfix<int8_t>(int8_t q, int shift) { return (int64_t)q * (1ll << shift); }
template <> __device__ __forceinline__ int64_t qfix<int32_t>(int32_t q, int shift) { return (int64_t)q * (1ll << shift); }
// q 2^S is exact in float (a power-of-two scaling that stays below 2^62), so
// the rounding to an integer is the same as in double, without FP64 arithmetic
template <> __device__ __forceinline__ int64_t qfix<float>(float q, int shift) {
    if (shift <= 100) return __float2ll_rn(q * ldexpf(1.0f, shift));
    return __double2ll_rn((double)q * ldexp(1.0, shift));
}
template <> __device__ __forceinline__ int64_t qfix<double>(double q, int shift) {
    return __double2ll_rn(q * ldexp(1.0, shift));
}

}  // namespace vqd
