// vq_resident.cu -- plan and launch of the resident kernel (the whole run of
// a sparse instance in one launch; kernel in vq_resident_kernel.cuh).
#include <algorithm>

#include "vq_resident_kernel.cuh"

namespace vq {

namespace {

using namespace resident;

KFn pick_kernel(int rc, int rpt, bool csr_smem, bool packed, int ell, int threads, int method) {
#define VQ_PICK_RC(M)                                                           \
    switch (rc) {                                                               \
        case 1: return resident_pick_rc1_m##M(rpt, csr_smem, packed, ell, threads); \
        case 2: return resident_pick_rc2_m##M(rpt, csr_smem, packed, ell, threads); \
        case 4: return resident_pick_rc4_m##M(rpt, csr_smem, packed, ell, threads); \
        default: return resident_pick_rc8_m##M(rpt, csr_smem, packed, ell, threads); \
    }
    if (method == VELOXQ_METHOD_PA) { VQ_PICK_RC(2) }
    if (method == VELOXQ_METHOD_ASB) { VQ_PICK_RC(1) }
    VQ_PICK_RC(0)
#undef VQ_PICK_RC
}

struct ResPlan {
    int rc, threads, rpt;
    bool csr_smem, packed;
    int ell_d;       // > 0: ELL layout with this many (even) slots per row
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
    const int sms = device_sms(ctx->device);
    ResPlan best{0, 0, 0, false, false, 0, 0, false};
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
        // ELL when the padded slots add at most a quarter to the couplings
        const int ell_d = ctx->max_row + (ctx->max_row & 1);
        const bool ell_ok = packed && ell_d > 0 && (double)ell_d * n <= 1.25 * (double)ctx->nnz + 2.0 * n;
        for (int cs = 2; cs >= 0; --cs) {
            const bool csr_smem = cs >= 1 && ctx->n <= 65535;
            const bool ell = cs == 2 && ell_ok;
            if (cs >= 1 && !csr_smem) continue;
            if (cs == 2 && !ell) continue;
            const SmemPlan p = plan_smem(n, csr_smem ? ctx->nnz : 0, rc, threads, nwords, csr_smem, csr_smem && packed,
                                         ell ? ell_d : 0);
            if (p.total > (size_t)kSmemMax) continue;
            const int64_t ctas = div_up(R, rc);
            const double cost = (double)div_up(ctas, sms) * (3.0 + rc) * (csr_smem ? 1.0 : 1.3);
            if (cost < best_cost - 1e-9) {
                best_cost = cost;
                best = ResPlan{rc, threads, rpt, csr_smem, csr_smem && packed, ell ? ell_d : 0, p.total, true};
            }
            break;   // the most compact variant that fits is preferred for this rc
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

bool resident_on_chip(const veloxq_ctx* ctx, int32_t R) {
    const ResPlan p = make_plan(ctx, R);
    return p.ok && p.csr_smem;
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
    a.ell_d = p.ell_d;
    a.method = rp.method;
    a.alpha = rp.alpha;
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
    KFn fn = pick_kernel(p.rc, p.rpt, p.csr_smem, p.packed, p.ell_d, p.threads, rp.method);
    if (!fn) return fail(VELOXQ_EUNSUPPORTED, "no resident kernel variant for this plan");
    VQ_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    fn<<<(unsigned)div_up(R, p.rc), p.threads, p.smem, ctx->stream>>>(a);
    VQ_LAUNCH_CHECK("resident kernel");
    return VELOXQ_OK;
}

}  // namespace vq
