// vq_api.cu -- the C ABI declared in include/veloxq.h: argument checks,
// context lifetime, path selection, the solve driver (CUDA-graph captured
// step loops or a single resident launch) and host <-> device marshalling.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "vq_internal.cuh"

namespace vq {

namespace {
thread_local std::string g_err;
}

void set_error(const std::string& msg) { g_err = msg; }

int fail(int status, const std::string& msg) {
    g_err = msg;
    return status;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    cudaGetLastError();   // a non-sticky error must not resurface in a later launch check
    if (e == cudaErrorMemoryAllocation) return VELOXQ_ENOMEM;
    return VELOXQ_ECUDA;
}

// ---------------------------------------------------------------------------
// Cache of released device blocks. Creating a context, solving on it and
// destroying it allocates and frees some twenty buffers; cudaMalloc and
// cudaFree of large blocks cost 0.1-0.35 ms each (page mapping), as much as a
// short solve. Released blocks are kept per device, up to a bounded total, and
// handed to the next request they fit (at most 1/4 + 64 KiB larger). A block
// enters the cache only after the device has finished all work issued so far
// (the wait cudaFree would do), so a later owner never races a kernel of the
// previous one. When an allocation fails, the device's cached blocks are freed
// and the allocation is tried once more.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kCacheMaxBytes = size_t(8) << 30;     // per device

struct BlockCache {
    std::mutex mu;
    std::map<int, std::multimap<size_t, void*>> free_blocks;   // device -> size -> block
    std::map<int, size_t> cached;                             // device -> bytes held
};

BlockCache& block_cache() {
    static BlockCache* c = new BlockCache();   // never destroyed: blocks go with the process
    return *c;
}

bool cache_enabled() {
    static const bool on = [] {
        const char* v = std::getenv("VELOXQ_ALLOC_CACHE");
        return !(v && v[0] == '0');
    }();
    return on;
}

void* cache_take(int dev, size_t b, size_t* got) {
    if (!cache_enabled()) return nullptr;
    BlockCache& c = block_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    auto& m = c.free_blocks[dev];
    auto it = m.lower_bound(b);
    if (it == m.end() || it->first > b + b / 4 + (size_t(64) << 10)) return nullptr;
    void* p = it->second;
    *got = it->first;
    c.cached[dev] -= it->first;
    m.erase(it);
    return p;
}

void cache_trim(int dev) {
    BlockCache& c = block_cache();
    std::vector<void*> out;
    {
        std::lock_guard<std::mutex> lk(c.mu);
        for (auto& kv : c.free_blocks[dev]) out.push_back(kv.second);
        c.free_blocks[dev].clear();
        c.cached[dev] = 0;
    }
    for (void* q : out) cudaFree(q);
}
}  // namespace

void DevBuf::release() {
    if (!p) return;
    bool kept = false;
    int cur = -1;
    if (cache_enabled() && cudaGetDevice(&cur) == cudaSuccess && cur == dev &&
        cudaDeviceSynchronize() == cudaSuccess) {
        BlockCache& c = block_cache();
        std::lock_guard<std::mutex> lk(c.mu);
        if (c.cached[dev] + bytes <= kCacheMaxBytes) {
            c.free_blocks[dev].emplace(bytes, p);
            c.cached[dev] += bytes;
            kept = true;
        }
    }
    if (!kept) cudaFree(p);
    p = nullptr;
    bytes = 0;
    dev = -1;
}

int DevBuf::ensure(size_t b) {
    if (b <= bytes && p) return VELOXQ_OK;
    release();
    if (b == 0) b = 16;
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e == cudaSuccess) {
        size_t got = 0;
        if (void* q = cache_take(d, b, &got)) {
            p = q;
            bytes = got;
            dev = d;
            return VELOXQ_OK;
        }
        e = cudaMalloc(&p, b);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            cache_trim(d);
            e = cudaMalloc(&p, b);
        }
    }
    if (e != cudaSuccess) {
        p = nullptr;
        bytes = 0;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? VELOXQ_ENOMEM : VELOXQ_ECUDA,
                    std::string("device allocation of ") + std::to_string(b) + " bytes failed: " + cudaGetErrorString(e));
    }
    bytes = b;
    dev = d;
    return VELOXQ_OK;
}

// extra per-context state kept out of the public struct definition
struct CtxExtra {
    cudaStream_t work = nullptr;
    cudaEvent_t ev = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr, t2 = nullptr, t3 = nullptr;   // timing of the last solve
    std::vector<uint64_t> graph_key;
    cudaGraphExec_t graph = nullptr;
    int64_t graph_launches = 0;
    veloxq_timing timing{};
    bool timed = false;
    // scratch of a batched launch headed by this context (instance table,
    // per-instance results, error word): owned here, so that batches headed
    // by different contexts never share it
    DevBuf bwork, bbest, berr;
    int tune_stages = 0, tune_split = 0;   // form of the last batched launch headed by this context
    BatchGraph bgraph;                     // its captured device part
    ~CtxExtra() {
        if (graph) cudaGraphExecDestroy(graph);
        for (cudaEvent_t e : {ev, t0, t1, t2, t3})
            if (e) cudaEventDestroy(e);
        if (work) cudaStreamDestroy(work);
    }
};

// The extra state of every live context, keyed by the context. Contexts are
// created and destroyed from any thread, so the map is only touched under its
// lock; an entry lives as long as its context.
std::mutex& extras_mu() {
    static std::mutex mu;
    return mu;
}
std::map<const veloxq_ctx*, std::unique_ptr<CtxExtra>>& extras() {
    static std::map<const veloxq_ctx*, std::unique_ptr<CtxExtra>> m;
    return m;
}

CtxExtra* extra(const veloxq_ctx* ctx) {
    std::lock_guard<std::mutex> lk(extras_mu());
    auto it = extras().find(ctx);
    return it == extras().end() ? nullptr : it->second.get();
}

int resolve(const veloxq_ctx* ctx, const veloxq_schedule* s_in, int32_t K, RunParams* p) {
    veloxq_schedule s;
    veloxq_schedule_default(&s);
    if (s_in) s = *s_in;
    if (!(std::isfinite(s.dt) && s.dt > 0)) return fail(VELOXQ_EINVAL, "schedule dt must be finite and > 0");
    if (!(std::isfinite(s.a0) && s.a0 > 0)) return fail(VELOXQ_EINVAL, "schedule a0 must be finite and > 0");
    if (!std::isfinite(s.kappa)) return fail(VELOXQ_EINVAL, "schedule kappa must be finite");
    if (!(std::isfinite(s.c0) && s.c0 >= 0)) return fail(VELOXQ_EINVAL, "schedule c0 must be finite and >= 0");
    if (!(std::isfinite(s.sigma0) && s.sigma0 >= 0)) return fail(VELOXQ_EINVAL, "schedule sigma0 must be finite and >= 0");
    if (s.n_knots < 0 || (s.n_knots > 0 && !s.a_knots)) return fail(VELOXQ_EINVAL, "schedule knots: n_knots < 0 or a_knots NULL");
    if (s.readout_every < 0) return fail(VELOXQ_EINVAL, "schedule readout_every must be >= 0");
    if (s.prec < VELOXQ_PREC_FP32 || s.prec > VELOXQ_PREC_FP8_ONE_TERM) return fail(VELOXQ_EINVAL, "unknown precision");
    if (s.path < VELOXQ_PATH_AUTO || s.path > VELOXQ_PATH_DENSE) return fail(VELOXQ_EINVAL, "unknown path");
    if (s.method < VELOXQ_METHOD_BSB || s.method > VELOXQ_METHOD_PA) return fail(VELOXQ_EINVAL, "unknown method");
    if (!(std::isfinite(s.momentum) && s.momentum >= 0 && s.momentum < 1))
        return fail(VELOXQ_EINVAL, "schedule momentum must be in [0, 1)");
    if (s.method == VELOXQ_METHOD_ASB && (s.prec == VELOXQ_PREC_FP8 || s.prec == VELOXQ_PREC_FP8_ONE_TERM))
        return fail(VELOXQ_EUNSUPPORTED, "adiabatic SB leaves [-1, 1]: no FP8 operand with a fixed scale");
    p->dt = s.dt;
    p->a0 = s.a0;
    p->sigma0 = s.sigma0;
    p->kappa = s.kappa;
    p->c0_given = s.c0 > 0;
    // J = -Qoff/2 => rho(J) = rho(Qoff)/2 and c0 = kappa / rho(J)
    p->c0 = s.c0 > 0 ? s.c0 : (ctx->rho > 1e-12 ? (float)(2.0 * s.kappa / ctx->rho) : s.kappa);
    p->K = K;
    p->readout_every = s.readout_every;
    p->prec = s.prec;
    p->path = s.path;
    p->method = (int)s.method;
    p->alpha = s.momentum;
    p->knots.clear();
    if (s.n_knots > 0) {
        for (int j = 0; j < s.n_knots; ++j) {
            if (!std::isfinite(s.a_knots[j])) return fail(VELOXQ_EINVAL, "schedule knot is not finite");
            p->knots.push_back(s.a_knots[j]);
        }
    } else {
        p->knots = {0.0, (double)s.a0};
    }
    return VELOXQ_OK;
}

// a_k, k = 0..K-1: piecewise linear through evenly spread knots
std::vector<float> schedule_table(const RunParams& p) {
    std::vector<float> a((size_t)p.K);
    const int nk = (int)p.knots.size();
    for (int k = 0; k < p.K; ++k) {
        if (p.K == 1 || nk == 1) { a[k] = (float)p.knots[0]; continue; }
        const double t = (double)k * (double)(nk - 1) / (double)(p.K - 1);
        int j = (int)std::floor(t);
        if (j > nk - 2) j = nk - 2;
        const double w = t - (double)j;
        a[k] = (float)(p.knots[j] * (1.0 - w) + p.knots[j + 1] * w);
    }
    return a;
}

int upload_schedule(veloxq_ctx* ctx, const RunParams& p) {
    std::vector<float> a = schedule_table(p);
    VQ_TRY(ctx->a_table.ensure(sizeof(float) * a.size()));
    VQ_CUDA(cudaMemcpyAsync(ctx->a_table.p, a.data(), sizeof(float) * a.size(), cudaMemcpyHostToDevice, ctx->stream));
    // the host vector dies at return: make the copy complete first
    VQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return VELOXQ_OK;
}

veloxq_path choose_path(const veloxq_ctx* ctx, veloxq_path want, veloxq_prec prec, int32_t R) {
    if (want != VELOXQ_PATH_AUTO) return want;
    if (ctx->dense && prec != VELOXQ_PREC_FP32) return VELOXQ_PATH_DENSE;
    if (ctx->dense) return resident_fits(ctx, R, nullptr, nullptr, nullptr) ? VELOXQ_PATH_RESIDENT : VELOXQ_PATH_DENSE;
    // sparse: the resident kernel only when its couplings stay in shared
    // memory; when every CTA has to re-read them from L2 each step, the
    // streaming step is faster (Pegasus P_16: 84 against 29 us per step at
    // 1024 replicas, Zephyr Z_12: 228 against 29)
    return resident_on_chip(ctx, R) ? VELOXQ_PATH_RESIDENT : VELOXQ_PATH_STREAM;
}

int check_path(const veloxq_ctx* ctx, veloxq_path path, veloxq_prec prec, int32_t R) {
    if (path == VELOXQ_PATH_DENSE && !ctx->dense) return fail(VELOXQ_EUNSUPPORTED, "dense path requested for a sparse context");
    if ((path == VELOXQ_PATH_STREAM || path == VELOXQ_PATH_RESIDENT) && !ctx->has_csr)
        return fail(VELOXQ_EUNSUPPORTED, "sparse-row path requested for a dense context without CSR rows (n > 512)");
    if ((path == VELOXQ_PATH_STREAM || path == VELOXQ_PATH_RESIDENT) && prec != VELOXQ_PREC_FP32)
        return fail(VELOXQ_EUNSUPPORTED, "the sparse-row kernels run the field in FP32");
    if (path == VELOXQ_PATH_RESIDENT && !resident_fits(ctx, R, nullptr, nullptr, nullptr))
        return fail(VELOXQ_EUNSUPPORTED, "instance does not fit the resident kernel");
    if (prec != VELOXQ_PREC_FP32 && !ctx->dense)
        return fail(VELOXQ_EUNSUPPORTED, "sparse contexts run the field in FP32 (or exact int8)");
    return VELOXQ_OK;
}

// Tensor-core operands of one run: quantised Q, two S operand buffers (each
// holding `terms` planes), maps (ms_lo: the lo planes of two-term FP8).
struct TcRun {
    CUtensorMap mq, ms[2], ms_lo[2];
    void* sop[2];
    int terms = 1;
    const CUtensorMap* lo() const { return terms == 2 ? ms_lo : nullptr; }
    const CUtensorMap* lo(int c) const { return terms == 2 ? &ms_lo[c] : nullptr; }
};

int tc_setup(veloxq_ctx* ctx, int prec, int32_t R, TcRun* t, int method = VELOXQ_METHOD_BSB) {
    VQ_TRY(tc_prepare_q(ctx, prec));
    t->terms = tc_terms(prec, method);
    const size_t b = tc_sop_bytes(ctx, prec, t->terms, R);
    VQ_TRY(ctx->sop_a.ensure(b));
    VQ_TRY(ctx->sop_b.ensure(b));
    VQ_TRY(ctx->errw.ensure(sizeof(int) * 4));
    // completion counters of multi-step runs, one per replica column block (sized before any capture)
    VQ_TRY(ctx->tcdone.ensure(sizeof(uint32_t) * (size_t)div_up(R, 256)));
    // the K padding columns [n, n_pad) of both operand buffers must stay zero:
    // the epilogue never writes them
    VQ_CUDA(cudaMemsetAsync(ctx->sop_a.p, 0, b, ctx->stream));
    VQ_CUDA(cudaMemsetAsync(ctx->sop_b.p, 0, b, ctx->stream));
    ctx->sop_tag = 0;
    t->sop[0] = ctx->sop_a.p;
    t->sop[1] = ctx->sop_b.p;
    return tc_maps(ctx, prec, t->terms, R, t->sop[0], t->sop[1], &t->mq, &t->ms[0], &t->ms[1], &t->ms_lo[0],
                   &t->ms_lo[1]);
}

// ---- autotuned form of the batched launch ---------------------------------
// Key of a batch kind: the device (name and SM count, so that a kept cache
// carries over to another machine with the same GPU), the field precision and
// integrator, the replicas, the instance count rounded up to a power of two,
// and the mean and largest n rounded up to multiples of 128.
std::string tune_key(const veloxq_ctx* c0, veloxq_ctx* const* ctxs, int32_t count, int32_t R, const RunParams& p) {
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, c0->device) != cudaSuccess) {
        cudaGetLastError();
        prop.name[0] = 0;
    }
    int64_t sum = 0, mx = 0;
    for (int32_t m = 0; m < count; ++m) {
        sum += ctxs[m]->n;
        mx = std::max<int64_t>(mx, ctxs[m]->n);
    }
    int64_t cnt = 1;
    while (cnt < count) cnt <<= 1;
    const int64_t mean = div_up(div_up(sum, std::max(1, count)), 128) * 128;
    std::string k = "batch|" + std::string(prop.name) + "|" + std::to_string(prop.multiProcessorCount) + "|prec" +
                    std::to_string((int)p.prec) + "|m" + std::to_string(p.method) + "|R" + std::to_string(R) + "|c" +
                    std::to_string(cnt) + "|nmean" + std::to_string(mean) + "|nmax" +
                    std::to_string(div_up(mx, 128) * 128);
    for (char& ch : k)
        if (ch == ' ' || ch == '=' || ch == '\n') ch = '_';
    return k;
}

namespace {
std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune;   // key -> (stages, replicas per work item)
bool g_tune_loaded = false;

// Lines "key=stages group" of the file VELOXQ_TUNE_CACHE names (read once).
void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = std::getenv("VELOXQ_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[1024];
    while (std::fgets(line, sizeof(line), f)) {
        char* eq = std::strchr(line, '=');
        if (!eq) continue;
        *eq = 0;
        int st = 0, grp = 0;
        if (std::sscanf(eq + 1, "%d %d", &st, &grp) == 2 && (st == 4 || st == 6) && grp >= 16 && grp % 16 == 0)
            g_tune[line] = {st, grp};
    }
    std::fclose(f);
}
}  // namespace

bool tune_lookup(const std::string& key, int* stages, int* group) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it == g_tune.end()) return false;
    *stages = it->second.first;
    *group = it->second.second;
    return true;
}

void tune_store(const std::string& key, int stages, int group) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    g_tune[key] = {stages, group};
    const char* path = std::getenv("VELOXQ_TUNE_CACHE");
    if (!path || !*path) return;
    if (FILE* f = std::fopen(path, "a")) {
        std::fprintf(f, "%s=%d %d\n", key.c_str(), stages, group);
        std::fclose(f);
    }
}

// Every call on a context runs on the device the context was created on,
// which must be the current device: its buffers live there.
int check_device(const veloxq_ctx* ctx) {
    int dev = -1;
    VQ_CUDA(cudaGetDevice(&dev));
    if (dev != ctx->device)
        return fail(VELOXQ_EINVAL, "the context was created on device " + std::to_string(ctx->device) +
                                       ", which must be the current device (current: " + std::to_string(dev) + ")");
    return VELOXQ_OK;
}

int check_err_word(veloxq_ctx* ctx) {
    int h = 0;
    VQ_CUDA(cudaMemcpyAsync(&h, ctx->errw.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    VQ_CUDA(cudaStreamSynchronize(ctx->stream));
    if (h) return fail(VELOXQ_ETIMEDOUT, "a bounded device wait in the tensor-core kernel gave up (code " +
                                             std::to_string(h) + ")");
    return VELOXQ_OK;
}

bool is_readout(const RunParams& p, int k) {
    return (k == p.K - 1) || (p.readout_every > 0 && ((k + 1) % p.readout_every) == 0);
}

// Enqueue the step loop (steps, readouts, argmin) on ctx->stream; ev_steps
// (if not null) is recorded right after the last integration step; tc_energy:
// readout energies in the tensor-core form (sized before the capture).
int enqueue_loop(veloxq_ctx* ctx, veloxq_path path, int32_t R, const RunParams& p, int nparts, const TcRun* tc,
                 bool tc_energy, cudaEvent_t ev_steps) {
    const Layout lay = path == VELOXQ_PATH_DENSE ? LAYOUT_RN : LAYOUT_NR;
    float* cur = ctx->s_a.as<float>();
    float* nxt = ctx->s_b.as<float>();
    float* Y = ctx->y.as<float>();
    const float* at = ctx->a_table.as<float>();
    int np = nparts;
    int cb = 0;   // tensor-core path: the operand of the next step is in sop[cb]
    for (int k = 0; k < p.K; ++k) {
        if (tc) {
            // every step up to the next readout in one launch
            int k1 = k;
            while (!is_readout(p, k1)) ++k1;
            VQ_TRY(tc_run(ctx, p.prec, R, tc->mq, tc->ms, tc->lo(), cb, cur, nxt, Y, tc->sop, at, k, k1 + 1, p.dt,
                          p.a0, p.c0, nullptr, ctx->errw.as<int>(), rule_of(p)));
            const int L = k1 + 1 - k;
            if (L & 1) {
                std::swap(cur, nxt);
                cb ^= 1;
            }
            k = k1;
        } else if (path == VELOXQ_PATH_DENSE) {
            VQ_TRY(dense_step(ctx, R, cur, nxt, Y, at, k, p.dt, p.a0, p.c0, nullptr, rule_of(p)));
        } else {
            VQ_TRY(stream_step(ctx, R, cur, nxt, Y, at, k, p.dt, p.a0, p.c0, nullptr, rule_of(p)));
        }
        if (!tc) std::swap(cur, nxt);
        // an event node of the graph (a plain record during capture would only order streams)
        if (ev_steps && k == p.K - 1) VQ_CUDA(cudaEventRecordWithFlags(ev_steps, ctx->stream, cudaEventRecordExternal));
        if (!is_readout(p, k)) continue;
        int64_t* parts = ctx->ework.as<int64_t>();
        if (path == VELOXQ_PATH_DENSE) VQ_TRY(dense_energy(ctx, R, cur, parts, &np, tc_energy));
        else VQ_TRY(stream_energy(ctx, R, cur, parts, &np));
        VQ_TRY(launch_best_update(ctx, R, np, parts, ctx->best_e.as<int64_t>(), ctx->flags.as<uint8_t>()));
        VQ_TRY(launch_best_bits(ctx, R, lay, cur, ctx->flags.as<uint8_t>(), ctx->best_bits.as<uint32_t>()));
    }
    VQ_TRY(launch_argmin_unpack(ctx, R, ctx->best_e.as<int64_t>(), ctx->best_bits.as<uint32_t>(),
                                ctx->misc.as<int64_t>(), ctx->xout.as<uint8_t>()));
    return VELOXQ_OK;
}

int stream_energy_parts_count(veloxq_ctx* ctx, veloxq_path path, int32_t R);

}  // namespace vq

// ---- forward declaration from vq_stream.cu
namespace vq {
int stream_energy_parts(int32_t R);
int stream_energy_parts_count(veloxq_ctx* ctx, veloxq_path path, int32_t R) {
    return path == VELOXQ_PATH_DENSE ? (int)div_up(ctx->n, 64) : stream_energy_parts(R);
}
}  // namespace vq

using namespace vq;

// Replica counts above 2^20 would overflow the second grid axis of the dense
// kernels (R / 32 blocks); no workload comes near it.
static constexpr int32_t kMaxReplicas = 1 << 20;

extern "C" {

void veloxq_schedule_default(veloxq_schedule* s) {
    if (!s) return;
    s->dt = 0.5f;
    s->a0 = 1.0f;
    s->kappa = 1.0f;
    s->c0 = 0.0f;
    s->sigma0 = 0.1f;
    s->n_knots = 0;
    s->a_knots = nullptr;
    s->readout_every = 50;
    s->prec = VELOXQ_PREC_FP32;
    s->path = VELOXQ_PATH_AUTO;
    s->method = VELOXQ_METHOD_BSB;
    s->momentum = 0.9f;
}

const char* veloxq_last_error(void) { return g_err.c_str(); }

static int new_ctx(veloxq_ctx** out, int64_t n, void* stream, veloxq_ctx** made) {
    if (!out) return fail(VELOXQ_EINVAL, "out must not be NULL");
    *out = nullptr;
    if (n < 1) return fail(VELOXQ_EINVAL, "n must be >= 1");
    if (n > ((int64_t)1 << 31) - 2) return fail(VELOXQ_EINVAL, "n must be < 2^31 - 1");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice (no CUDA device?)");
    veloxq_ctx* ctx = new (std::nothrow) veloxq_ctx();
    if (!ctx) return fail(VELOXQ_ENOMEM, "host allocation failed");
    ctx->device = dev;
    ctx->stream = (cudaStream_t)stream;
    ctx->n = n;
    auto ex = std::make_unique<CtxExtra>();
    e = cudaStreamCreateWithFlags(&ex->work, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ex->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&ex->t0);
    if (e == cudaSuccess) e = cudaEventCreate(&ex->t1);
    if (e == cudaSuccess) e = cudaEventCreate(&ex->t2);
    if (e == cudaSuccess) e = cudaEventCreate(&ex->t3);
    if (e != cudaSuccess) {
        delete ctx;
        return cuda_fail(e, "stream creation");
    }
    {
        std::lock_guard<std::mutex> lk(extras_mu());
        extras()[ctx] = std::move(ex);
    }
    *made = ctx;
    return VELOXQ_OK;
}

static int finish_ctx(veloxq_ctx* ctx, int st, veloxq_ctx** out) {
    if (st == VELOXQ_OK) st = power_iteration(ctx, 300, &ctx->rho);
    if (st != VELOXQ_OK) {
        std::string keep = g_err;
        veloxq_destroy(ctx);
        g_err = keep;
        return st;
    }
    *out = ctx;
    return VELOXQ_OK;
}

int veloxq_create_dense(veloxq_ctx** out, int64_t n, veloxq_vtype vt, const void* Q, const double* c, void* stream) {
    if (!Q) return fail(VELOXQ_EINVAL, "Q must not be NULL");
    if (n > (1 << 20)) return fail(VELOXQ_EINVAL, "dense n must be <= 2^20");
    veloxq_ctx* ctx = nullptr;
    VQ_TRY(new_ctx(out, n, stream, &ctx));
    return finish_ctx(ctx, ingest_dense(ctx, vt, Q, c, false), out);
}

int veloxq_create_ising_dense(veloxq_ctx** out, int64_t n, veloxq_vtype vt, const void* J, const double* h, void* stream) {
    if (!J) return fail(VELOXQ_EINVAL, "J must not be NULL");
    if (n > (1 << 20)) return fail(VELOXQ_EINVAL, "dense n must be <= 2^20");
    veloxq_ctx* ctx = nullptr;
    VQ_TRY(new_ctx(out, n, stream, &ctx));
    return finish_ctx(ctx, ingest_dense(ctx, vt, J, h, true), out);
}

int veloxq_create_csr(veloxq_ctx** out, int64_t n, const int64_t* rowptr, const int32_t* col, veloxq_vtype vt,
                      const void* val, const double* c, void* stream) {
    if (!rowptr) return fail(VELOXQ_EINVAL, "rowptr must not be NULL");
    veloxq_ctx* ctx = nullptr;
    VQ_TRY(new_ctx(out, n, stream, &ctx));
    return finish_ctx(ctx, ingest_csr(ctx, rowptr, col, vt, val, c, false), out);
}

int veloxq_create_ising_csr(veloxq_ctx** out, int64_t n, const int64_t* rowptr, const int32_t* col, veloxq_vtype vt,
                            const void* J, const double* h, void* stream) {
    if (!rowptr) return fail(VELOXQ_EINVAL, "rowptr must not be NULL");
    veloxq_ctx* ctx = nullptr;
    VQ_TRY(new_ctx(out, n, stream, &ctx));
    return finish_ctx(ctx, ingest_csr(ctx, rowptr, col, vt, J, h, true), out);
}

void veloxq_destroy(veloxq_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    std::unique_ptr<CtxExtra> gone;
    {
        std::lock_guard<std::mutex> lk(extras_mu());
        auto it = extras().find(ctx);
        if (it != extras().end()) {
            gone = std::move(it->second);
            extras().erase(it);
        }
    }
    gone.reset();
    delete ctx;
}

int veloxq_get_info(veloxq_ctx* ctx, veloxq_info* info) {
    if (!ctx || !info) return fail(VELOXQ_EINVAL, "ctx and info must not be NULL");
    info->n = ctx->n;
    info->nnz_field = ctx->nnz;
    info->is_dense = ctx->dense ? 1 : 0;
    info->is_integer = ctx->integer ? 1 : 0;
    info->rho = ctx->rho;
    info->K0 = ctx->K0;
    info->ising_offset = ctx->ising_offset;
    return VELOXQ_OK;
}

int veloxq_set_stream(veloxq_ctx* ctx, void* stream) {
    if (!ctx) return fail(VELOXQ_EINVAL, "ctx must not be NULL");
    ctx->stream = (cudaStream_t)stream;
    return VELOXQ_OK;
}

int veloxq_last_timing(veloxq_ctx* ctx, veloxq_timing* timing) {
    if (!ctx || !timing) return fail(VELOXQ_EINVAL, "ctx and timing must not be NULL");
    CtxExtra* ex = extra(ctx);
    if (!ex || !ex->timed) return fail(VELOXQ_EINVAL, "no solve has completed on this context");
    *timing = ex->timing;
    return VELOXQ_OK;
}

int veloxq_spectral_radius(veloxq_ctx* ctx, double* rho) {
    if (!ctx || !rho) return fail(VELOXQ_EINVAL, "ctx and rho must not be NULL");
    *rho = ctx->rho;
    return VELOXQ_OK;
}

int veloxq_solve(veloxq_ctx* ctx, int32_t replicas, int32_t steps, const veloxq_schedule* sched, uint64_t seed,
                 uint8_t* x_best, double* E_best, int64_t* E_best_int, double* E_per_replica) {
    if (!ctx) return fail(VELOXQ_EINVAL, "ctx must not be NULL");
    VQ_TRY(check_device(ctx));
    if (replicas < 1 || replicas > kMaxReplicas) return fail(VELOXQ_EINVAL, "replicas must be in [1, 2^20]");
    if (steps < 1) return fail(VELOXQ_EINVAL, "steps must be >= 1");
    if (E_best_int && !ctx->integer) return fail(VELOXQ_EINVAL, "E_best_int requires an integer-valued context");
    RunParams p;
    VQ_TRY(resolve(ctx, sched, steps, &p));
    const veloxq_path path = choose_path(ctx, p.path, p.prec, replicas);
    VQ_TRY(check_path(ctx, path, p.prec, replicas));
    ctx->batch_R = 0;
    CtxExtra* ex = extra(ctx);
    const int64_t n = ctx->n, R = replicas, nw = div_up(n, 32);
    // a NULL (legacy default) stream cannot be captured: run on the context's
    // private stream, ordered after it
    cudaStream_t user = ctx->stream;
    if (user == nullptr) {
        VQ_CUDA(cudaEventRecord(ex->ev, user));
        VQ_CUDA(cudaStreamWaitEvent(ex->work, ex->ev, 0));
        ctx->stream = ex->work;
    }
    struct Restore {
        veloxq_ctx* c;
        cudaStream_t s;
        ~Restore() { c->stream = s; }
    } restore{ctx, user};
    ex->timed = false;
    int64_t launches = 0;

    VQ_TRY(upload_schedule(ctx, p));
    VQ_TRY(ctx->best_e.ensure(sizeof(int64_t) * R));
    VQ_TRY(ctx->best_bits.ensure(sizeof(uint32_t) * R * nw));
    VQ_TRY(ctx->misc.ensure(sizeof(int64_t) * 16));
    VQ_TRY(ctx->xout.ensure((size_t)n));
    int32_t main_launches = 1;
    if (path == VELOXQ_PATH_RESIDENT) {
        VQ_CUDA(cudaEventRecord(ex->t0, ctx->stream));
        VQ_CUDA(cudaEventRecord(ex->t1, ctx->stream));
        VQ_TRY(resident_run(ctx, replicas, p, seed, 0, steps, nullptr, nullptr, nullptr, nullptr, nullptr,
                            ctx->best_e.as<int64_t>(), ctx->best_bits.as<uint32_t>()));
        VQ_CUDA(cudaEventRecord(ex->t2, ctx->stream));
        VQ_TRY(launch_argmin_unpack(ctx, replicas, ctx->best_e.as<int64_t>(), ctx->best_bits.as<uint32_t>(),
                                    ctx->misc.as<int64_t>(), ctx->xout.as<uint8_t>()));
        VQ_CUDA(cudaEventRecord(ex->t3, ctx->stream));
        launches = 3;
    } else {
        const Layout lay = path == VELOXQ_PATH_DENSE ? LAYOUT_RN : LAYOUT_NR;
        const int nparts = stream_energy_parts_count(ctx, path, replicas);
        VQ_TRY(ctx->s_a.ensure(sizeof(float) * n * R));
        VQ_TRY(ctx->s_b.ensure(sizeof(float) * n * R));
        VQ_TRY(ctx->y.ensure(sizeof(float) * n * R));
        VQ_TRY(ctx->ework.ensure(sizeof(int64_t) * (size_t)nparts * R));
        VQ_TRY(ctx->flags.ensure((size_t)R));
        if (path == VELOXQ_PATH_STREAM)
            VQ_TRY(stream_autotune(ctx, replicas, ctx->s_a.as<float>(), ctx->s_b.as<float>(), ctx->y.as<float>()));
        TcRun tc;
        const bool use_tc = path == VELOXQ_PATH_DENSE && p.prec != VELOXQ_PREC_FP32;
        if (use_tc) VQ_TRY(tc_setup(ctx, p.prec, replicas, &tc, p.method));
        if (path == VELOXQ_PATH_DENSE && !use_tc) VQ_TRY(dense_prepare(ctx, replicas));
        if (path == VELOXQ_PATH_DENSE) VQ_TRY(tc_energy_prepare(ctx, replicas));
        const bool tc_e = path == VELOXQ_PATH_DENSE && tc_energy_ready(ctx, replicas);
        VQ_CUDA(cudaEventRecord(ex->t0, ctx->stream));
        VQ_TRY(launch_init_state(ctx, replicas, seed, p.sigma0, lay, ctx->s_a.as<float>(), ctx->y.as<float>()));
        if (use_tc || tc_e) VQ_CUDA(cudaMemsetAsync(ctx->errw.p, 0, sizeof(int), ctx->stream));
        if (use_tc) VQ_TRY(tc_quant_s(ctx, p.prec, replicas, ctx->s_a.as<float>(), tc.sop[0], rule_of(p)));
        VQ_CUDA(cudaMemsetAsync(ctx->best_e.p, 0x7f, sizeof(int64_t) * R, ctx->stream));
        VQ_CUDA(cudaMemsetAsync(ctx->best_bits.p, 0, sizeof(uint32_t) * R * nw, ctx->stream));
        // the captured loop depends on every pointer and parameter below
        std::vector<uint64_t> key = {(uint64_t)path, (uint64_t)p.prec, (uint64_t)(uintptr_t)ctx->sop_a.p,
                                     (uint64_t)(uintptr_t)ctx->sop_b.p, (uint64_t)(uintptr_t)ctx->errw.p,
                                     (uint64_t)R, (uint64_t)steps, (uint64_t)p.readout_every,
                                     (uint64_t)(uintptr_t)ctx->s_a.p, (uint64_t)(uintptr_t)ctx->s_b.p,
                                     (uint64_t)(uintptr_t)ctx->y.p, (uint64_t)(uintptr_t)ctx->ework.p,
                                     (uint64_t)(uintptr_t)ctx->best_e.p, (uint64_t)(uintptr_t)ctx->best_bits.p,
                                     (uint64_t)(uintptr_t)ctx->flags.p, (uint64_t)(uintptr_t)ctx->misc.p,
                                     (uint64_t)(uintptr_t)ctx->xout.p, (uint64_t)(uintptr_t)ctx->a_table.p};
        key.push_back((uint64_t)p.method);
        for (uint64_t v : {(uint64_t)tc_e, (uint64_t)ctx->eplanes, (uint64_t)(uintptr_t)ctx->eplane.p,
                           (uint64_t)(uintptr_t)ctx->exop.p, (uint64_t)(uintptr_t)ctx->efield.p})
            key.push_back(v);
        float fp[4] = {p.dt, p.a0, p.c0, p.alpha};
        for (float f : fp) {
            uint32_t u;
            std::memcpy(&u, &f, 4);
            key.push_back(u);
        }
        if (!ex->graph || ex->graph_key != key) {
            if (ex->graph) {
                cudaGraphExecDestroy(ex->graph);
                ex->graph = nullptr;
            }
            cudaGraph_t g = nullptr;
            VQ_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            int st = enqueue_loop(ctx, path, replicas, p, nparts, use_tc ? &tc : nullptr, tc_e, ex->t2);
            cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
            if (st != VELOXQ_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (ce != cudaSuccess) return cuda_fail(ce, "graph capture");
            size_t nodes = 0;
            cudaGraphGetNodes(g, nullptr, &nodes);
            ce = cudaGraphInstantiate(&ex->graph, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) {
                ex->graph = nullptr;
                return cuda_fail(ce, "graph instantiate");
            }
            ex->graph_key = key;
            ex->graph_launches = (int64_t)nodes;
        }
        VQ_CUDA(cudaEventRecord(ex->t1, ctx->stream));
        VQ_CUDA(cudaGraphLaunch(ex->graph, ctx->stream));   // records t2 after the last step
        VQ_CUDA(cudaEventRecord(ex->t3, ctx->stream));
        launches = 1 + (use_tc ? 1 : 0) + ex->graph_launches;   // init (+ operand) kernels + graph nodes
        main_launches = steps;
        if (use_tc) {
            // one launch per run of steps up to a readout
            main_launches = 0;
            for (int k = 0; k < steps; ++k) main_launches += is_readout(p, k) ? 1 : 0;
        }
        if (use_tc || tc_e) VQ_TRY(check_err_word(ctx));
    }
    std::vector<int64_t> be((size_t)R);
    int64_t misc[2] = {0, 0};
    VQ_CUDA(cudaMemcpyAsync(be.data(), ctx->best_e.p, sizeof(int64_t) * R, cudaMemcpyDeviceToHost, ctx->stream));
    VQ_CUDA(cudaMemcpyAsync(misc, ctx->misc.p, sizeof(misc), cudaMemcpyDeviceToHost, ctx->stream));
    if (x_best) VQ_CUDA(cudaMemcpyAsync(x_best, ctx->xout.p, (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
    VQ_CUDA(cudaStreamSynchronize(ctx->stream));
    VQ_LAUNCH_CHECK("solve");
    {
        float a = 0.f, b = 0.f;
        VQ_CUDA(cudaEventElapsedTime(&a, ex->t0, ex->t3));
        VQ_CUDA(cudaEventElapsedTime(&b, ex->t1, ex->t2));
        ex->timing.ms_total = a;
        ex->timing.ms_main = b;
        ex->timing.launches = launches;
        ex->timing.path = (int32_t)path;
        ex->timing.main_launches = main_launches;
        const bool streamed = path == VELOXQ_PATH_STREAM;
        ex->timing.stream_gather = streamed ? ctx->stream_unroll : 0;
        ex->timing.stream_chunk = streamed ? ctx->stream_cvec * vec_width(replicas) : 0;
        ex->timing.batch_stages = 0;
        ex->timing.batch_group = 0;
        ex->timed = true;
    }
    const int sh = ctx->energy_shift;
    if (E_best) *E_best = std::ldexp((double)misc[1], -sh);
    if (E_best_int) *E_best_int = misc[1] >> sh;
    if (E_per_replica)
        for (int64_t r = 0; r < R; ++r) E_per_replica[r] = std::ldexp((double)be[r], -sh);
    return VELOXQ_OK;
}

int veloxq_solve_batch(veloxq_ctx* const* ctxs, int32_t count, int32_t replicas, int32_t steps,
                       const veloxq_schedule* sched, uint64_t seed, uint8_t* const* x_best, double* E_best) {
    if (count < 0 || (count > 0 && !ctxs)) return fail(VELOXQ_EINVAL, "ctxs must hold count contexts");
    if (count == 0) return VELOXQ_OK;
    if (replicas < 1 || replicas > kMaxReplicas || steps < 1)
        return fail(VELOXQ_EINVAL, "replicas must be in [1, 2^20] and steps >= 1");
    for (int32_t m = 0; m < count; ++m)
        if (!ctxs[m]) return fail(VELOXQ_EINVAL, "context " + std::to_string(m) + " is NULL");
    RunParams p;
    VQ_TRY(resolve(ctxs[0], sched, steps, &p));
    {
        int dev = 0;
        VQ_CUDA(cudaGetDevice(&dev));
        for (int32_t m = 0; m < count; ++m)
            if (ctxs[m]->device != dev)
                return fail(VELOXQ_EINVAL, "context " + std::to_string(m) + " was created on device " +
                                               std::to_string(ctxs[m]->device) + ", not the current device " +
                                               std::to_string(dev) + ": a batch runs on one device");
    }
    if (!batch_supported(ctxs, count, replicas, p)) {
        // general case: one solve per context
        for (int32_t m = 0; m < count; ++m) {
            int st = veloxq_solve(ctxs[m], replicas, steps, sched, seed, x_best ? x_best[m] : nullptr,
                                  E_best ? E_best + m : nullptr, nullptr, nullptr);
            if (st != VELOXQ_OK) return fail(st, "instance " + std::to_string(m) + ": " + g_err);
        }
        return VELOXQ_OK;
    }
    // one persistent launch for the whole batch, on the first context's private stream
    veloxq_ctx* c0 = ctxs[0];
    CtxExtra* ex = extra(c0);
    cudaStream_t st = ex->work;
    for (int32_t m = 0; m < count; ++m) {
        VQ_CUDA(cudaEventRecord(ex->ev, ctxs[m]->stream));
        VQ_CUDA(cudaStreamWaitEvent(st, ex->ev, 0));
    }
    {
        cudaStream_t keep = c0->stream;
        c0->stream = st;
        int rc = upload_schedule(c0, p);
        c0->stream = keep;
        VQ_TRY(rc);
    }
    DevBuf& work = ex->bwork;
    DevBuf& best_all = ex->bbest;
    DevBuf& errw = ex->berr;
    VQ_TRY(best_all.ensure(sizeof(int64_t) * 2 * (size_t)count));
    VQ_TRY(errw.ensure(sizeof(int) * 4));
    VQ_CUDA(cudaMemsetAsync(errw.p, 0, sizeof(int), st));
    // autotune the form of the launch: pipeline depth (4 stages at two CTAs
    // per SM, or 6 at one) and replicas per CTA (R, R/2, R/4: every work item a
    // replica group of an instance), by timing a probe of at most 2 steps of
    // every candidate; cached per device and batch kind (tune_key), shared by
    // every thread under a lock, and kept in the file VELOXQ_TUNE_CACHE names
    // (if set) for later processes
    const std::string key = tune_key(c0, ctxs, count, replicas, p);
    int stages = 0, split = 1;
    if (const char* form = std::getenv("VELOXQ_BATCH_FORM")) {
        // a form fixed by the caller: "stages group"
        int st2 = 0, grp = 0;
        if (std::sscanf(form, "%d %d", &st2, &grp) != 2 || (st2 != 4 && st2 != 6) || grp < 16 || grp % 16 != 0 ||
            replicas % grp != 0 || !batch_stages_fit(p.prec, p.method, st2, grp))
            return fail(VELOXQ_EINVAL, "VELOXQ_BATCH_FORM must be \"stages group\" with stages 4 or 6 and a group of "
                                       "16k replicas dividing the replica count that fits shared memory");
        stages = st2;
        split = replicas / grp;
    } else if (int grp = 0; tune_lookup(key, &stages, &grp) && grp <= replicas && replicas % grp == 0 &&
                            batch_stages_fit(p.prec, p.method, stages, grp)) {
        split = replicas / grp;
    } else {
        stages = 0;
        RunParams probe = p;
        probe.K = std::min(steps, 2);
        float best_ms = 1e30f;
        for (int sp : {1, 2, 4}) {
            if (replicas % sp != 0 || (replicas / sp) % 16 != 0) continue;
            for (int cand : {4, 6}) {
                if (!batch_stages_fit(p.prec, p.method, cand, replicas / sp)) continue;
                float ms = 0.f;
                VQ_TRY(batch_run(ctxs, count, replicas, probe, seed, st, cand, sp, work, best_all.as<int64_t>(),
                                 errw.as<int>(), &ms));
                if (ms < best_ms) {
                    best_ms = ms;
                    stages = cand;
                    split = sp;
                }
            }
        }
        if (!stages) return fail(VELOXQ_EUNSUPPORTED, "no batched form fits this replica count");
        tune_store(key, stages, replicas / split);
    }
    ex->tune_stages = stages;
    ex->tune_split = split;
    float ms_main = 0.f;
    int64_t nlaunch = 0;
    VQ_TRY(batch_run(ctxs, count, replicas, p, seed, st, stages, split, work, best_all.as<int64_t>(), errw.as<int>(),
                     &ms_main, &nlaunch, &ex->bgraph));
    int herr = 0;
    std::vector<int64_t> h((size_t)(2 * count));
    VQ_CUDA(cudaMemcpyAsync(&herr, errw.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    VQ_CUDA(cudaMemcpyAsync(h.data(), best_all.p, sizeof(int64_t) * h.size(), cudaMemcpyDeviceToHost, st));
    for (int32_t m = 0; m < count; ++m)
        if (x_best && x_best[m])
            VQ_CUDA(cudaMemcpyAsync(x_best[m], ctxs[m]->xout.p, (size_t)ctxs[m]->n, cudaMemcpyDeviceToHost, st));
    VQ_CUDA(cudaStreamSynchronize(st));
    if (herr) return fail(VELOXQ_ETIMEDOUT, "a bounded wait in the batched kernel gave up (code " + std::to_string(herr) + ")");
    if (E_best)
        for (int32_t m = 0; m < count; ++m) E_best[m] = std::ldexp((double)h[2 * m + 1], -ctxs[m]->energy_shift);
    ex->timing.ms_total = ms_main;
    ex->timing.ms_main = ms_main;
    ex->timing.launches = nlaunch;
    ex->timing.path = VELOXQ_PATH_DENSE;
    ex->timing.main_launches = 1;
    ex->timing.stream_gather = 0;
    ex->timing.stream_chunk = 0;
    ex->timing.batch_stages = stages;
    ex->timing.batch_group = replicas / split;
    ex->timed = true;
    return VELOXQ_OK;
}

// allow_tc: a dense context may take the tensor-core form, whose bounded
// waits are checked here (this synchronises the stream)
static int energy_impl(veloxq_ctx* ctx, int64_t B, const uint8_t* Xd, double* Ed, int64_t* Eid, bool allow_tc) {
    int64_t* parts;
    int np = 0;
    const int64_t chunk = 65535;
    bool tc_e = false;
    if (allow_tc && ctx->dense && B > 0) {
        VQ_TRY(tc_energy_prepare(ctx, std::min(chunk, B)));
        tc_e = tc_energy_ready(ctx, std::min(chunk, B));
        if (tc_e) VQ_CUDA(cudaMemsetAsync(ctx->errw.p, 0, sizeof(int), ctx->stream));
    }
    for (int64_t b0 = 0; b0 < B; b0 += chunk) {
        const int64_t nb = std::min(chunk, B - b0);
        const int npmax = ctx->dense ? (int)div_up(ctx->n, 64) : 64;
        VQ_TRY(ctx->ework.ensure(sizeof(int64_t) * (size_t)npmax * nb));
        parts = ctx->ework.as<int64_t>();
        if (ctx->dense) VQ_TRY(dense_energy_x(ctx, nb, Xd + b0 * ctx->n, parts, &np, tc_e));
        else VQ_TRY(sparse_energy_x(ctx, nb, Xd + b0 * ctx->n, parts, &np));
        VQ_TRY(launch_sum_parts(ctx, nb, np, parts, Ed ? Ed + b0 : nullptr, Eid ? Eid + b0 : nullptr));
    }
    if (tc_e) VQ_TRY(check_err_word(ctx));
    return VELOXQ_OK;
}

int veloxq_energy_dev(veloxq_ctx* ctx, int64_t batch, const uint8_t* X, double* E, int64_t* E_int) {
    if (!ctx) return fail(VELOXQ_EINVAL, "ctx must not be NULL");
    VQ_TRY(check_device(ctx));
    if (batch < 0) return fail(VELOXQ_EINVAL, "batch must be >= 0");
    if (batch > 0 && !X) return fail(VELOXQ_EINVAL, "X must not be NULL");
    if (E_int && !ctx->integer) return fail(VELOXQ_EINVAL, "E_int requires an integer-valued context");
    return energy_impl(ctx, batch, X, E, E_int, false);
}

int veloxq_energy(veloxq_ctx* ctx, int64_t batch, const uint8_t* X, double* E, int64_t* E_int) {
    if (!ctx) return fail(VELOXQ_EINVAL, "ctx must not be NULL");
    VQ_TRY(check_device(ctx));
    if (batch < 0) return fail(VELOXQ_EINVAL, "batch must be >= 0");
    if (batch > 0 && !X) return fail(VELOXQ_EINVAL, "X must not be NULL");
    if (E_int && !ctx->integer) return fail(VELOXQ_EINVAL, "E_int requires an integer-valued context");
    if (batch == 0) return VELOXQ_OK;
    DevBuf xd, ed, eid;
    VQ_TRY(xd.ensure((size_t)(batch * ctx->n)));
    VQ_TRY(ed.ensure(sizeof(double) * batch));
    if (E_int) VQ_TRY(eid.ensure(sizeof(int64_t) * batch));
    VQ_CUDA(cudaMemcpyAsync(xd.p, X, (size_t)(batch * ctx->n), cudaMemcpyHostToDevice, ctx->stream));
    VQ_TRY(energy_impl(ctx, batch, xd.as<uint8_t>(), ed.as<double>(), E_int ? eid.as<int64_t>() : nullptr, true));
    if (E) VQ_CUDA(cudaMemcpyAsync(E, ed.p, sizeof(double) * batch, cudaMemcpyDeviceToHost, ctx->stream));
    if (E_int) VQ_CUDA(cudaMemcpyAsync(E_int, eid.p, sizeof(int64_t) * batch, cudaMemcpyDeviceToHost, ctx->stream));
    VQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return VELOXQ_OK;
}

int veloxq_batch_state_dev(veloxq_ctx* ctx, int32_t R, float* S, float* Y) {
    if (!ctx || !S || !Y) return fail(VELOXQ_EINVAL, "ctx, S and Y must not be NULL");
    VQ_TRY(check_device(ctx));
    if (ctx->batch_R != R || R < 1) return fail(VELOXQ_EINVAL, "no batched state held for this replica count");
    const size_t b = sizeof(float) * (size_t)(ctx->n * (int64_t)R);
    VQ_CUDA(cudaMemcpyAsync(S, ctx->s_a.p, b, cudaMemcpyDeviceToDevice, ctx->stream));
    VQ_CUDA(cudaMemcpyAsync(Y, ctx->y.p, b, cudaMemcpyDeviceToDevice, ctx->stream));
    return VELOXQ_OK;
}

int veloxq_init_state_dev(veloxq_ctx* ctx, int32_t R, uint64_t seed, float sigma0, float* S, float* Y) {
    if (!ctx) return fail(VELOXQ_EINVAL, "ctx must not be NULL");
    VQ_TRY(check_device(ctx));
    if (R < 1 || R > kMaxReplicas || !S || !Y) return fail(VELOXQ_EINVAL, "R in [1, 2^20] and non-NULL S, Y required");
    if (!(std::isfinite(sigma0) && sigma0 >= 0)) return fail(VELOXQ_EINVAL, "sigma0 must be finite and >= 0");
    return launch_init_state(ctx, R, seed, sigma0, LAYOUT_RN, S, Y);
}

int veloxq_field_dev(veloxq_ctx* ctx, int32_t R, veloxq_prec prec, const float* S, float* F) {
    if (!ctx) return fail(VELOXQ_EINVAL, "ctx must not be NULL");
    VQ_TRY(check_device(ctx));
    if (R < 1 || R > kMaxReplicas || !S || !F) return fail(VELOXQ_EINVAL, "R in [1, 2^20] and non-NULL S, F required");
    if (prec < VELOXQ_PREC_FP32 || prec > VELOXQ_PREC_FP8_ONE_TERM) return fail(VELOXQ_EINVAL, "unknown precision");
    if (ctx->dense) {
        if (prec == VELOXQ_PREC_FP32) return dense_field(ctx, R, S, F);
        TcRun tc;
        VQ_TRY(tc_setup(ctx, prec, R, &tc));
        VQ_CUDA(cudaMemsetAsync(ctx->errw.p, 0, sizeof(int), ctx->stream));
        VQ_TRY(tc_quant_s(ctx, prec, R, S, tc.sop[0]));
        VQ_TRY(tc_field(ctx, prec, R, tc.mq, tc.ms[0], tc.lo(0), F, ctx->errw.as<int>()));
        return check_err_word(ctx);
    }
    if (prec != VELOXQ_PREC_FP32) return fail(VELOXQ_EUNSUPPORTED, "sparse contexts run the field in FP32 (or exact int8)");
    const int64_t nR = ctx->n * (int64_t)R;
    VQ_TRY(ctx->s_a.ensure(sizeof(float) * nR));
    VQ_TRY(ctx->f.ensure(sizeof(float) * nR));
    VQ_TRY(launch_transpose(ctx->stream, S, ctx->s_a.as<float>(), R, ctx->n));
    VQ_TRY(stream_field(ctx, R, ctx->s_a.as<float>(), ctx->f.as<float>()));
    return launch_transpose(ctx->stream, ctx->f.as<float>(), F, ctx->n, R);
}

int veloxq_steps_dev(veloxq_ctx* ctx, int32_t R, int32_t k_begin, int32_t k_count, int32_t K,
                     const veloxq_schedule* sched, float* S, float* Y, float* F_last) {
    if (!ctx) return fail(VELOXQ_EINVAL, "ctx must not be NULL");
    VQ_TRY(check_device(ctx));
    if (R < 1 || R > kMaxReplicas || !S || !Y) return fail(VELOXQ_EINVAL, "R in [1, 2^20] and non-NULL S, Y required");
    if (K < 1 || k_begin < 0 || k_count < 0 || (int64_t)k_begin + k_count > K)
        return fail(VELOXQ_EINVAL, "need 0 <= k_begin, 0 <= k_count, k_begin + k_count <= K");
    if (k_count == 0) return VELOXQ_OK;
    RunParams p;
    VQ_TRY(resolve(ctx, sched, K, &p));
    const veloxq_path path = choose_path(ctx, p.path, p.prec, R);
    VQ_TRY(check_path(ctx, path, p.prec, R));
    VQ_TRY(upload_schedule(ctx, p));
    const int64_t n = ctx->n, nR = n * (int64_t)R;
    const int k_end = k_begin + k_count;
    if (path == VELOXQ_PATH_RESIDENT)
        return resident_run(ctx, R, p, 0, k_begin, k_end, S, Y, S, Y, F_last, nullptr, nullptr);
    VQ_TRY(ctx->s_a.ensure(sizeof(float) * nR));
    VQ_TRY(ctx->s_b.ensure(sizeof(float) * nR));
    const float* at = ctx->a_table.as<float>();
    float* cur = ctx->s_a.as<float>();
    float* nxt = ctx->s_b.as<float>();
    if (path == VELOXQ_PATH_DENSE) {
        VQ_CUDA(cudaMemcpyAsync(cur, S, sizeof(float) * nR, cudaMemcpyDeviceToDevice, ctx->stream));
        if (p.prec != VELOXQ_PREC_FP32) {
            TcRun tc;
            VQ_TRY(tc_setup(ctx, p.prec, R, &tc, p.method));
            VQ_CUDA(cudaMemsetAsync(ctx->errw.p, 0, sizeof(int), ctx->stream));
            VQ_TRY(tc_quant_s(ctx, p.prec, R, cur, tc.sop[0], rule_of(p)));
            // the whole range in one launch (the solve's form)
            VQ_TRY(tc_run(ctx, p.prec, R, tc.mq, tc.ms, tc.lo(), 0, cur, nxt, Y, tc.sop, at, k_begin, k_end, p.dt,
                          p.a0, p.c0, F_last, ctx->errw.as<int>(), rule_of(p)));
            if (k_count & 1) std::swap(cur, nxt);
            VQ_CUDA(cudaMemcpyAsync(S, cur, sizeof(float) * nR, cudaMemcpyDeviceToDevice, ctx->stream));
            return check_err_word(ctx);
        }
        for (int k = k_begin; k < k_end; ++k) {
            VQ_TRY(dense_step(ctx, R, cur, nxt, Y, at, k, p.dt, p.a0, p.c0, k == k_end - 1 ? F_last : nullptr,
                              rule_of(p)));
            std::swap(cur, nxt);
        }
        VQ_CUDA(cudaMemcpyAsync(S, cur, sizeof(float) * nR, cudaMemcpyDeviceToDevice, ctx->stream));
        return VELOXQ_OK;
    }
    VQ_TRY(ctx->y.ensure(sizeof(float) * nR));
    VQ_TRY(ctx->f.ensure(sizeof(float) * nR));
    VQ_TRY(launch_transpose(ctx->stream, S, cur, R, n));
    VQ_TRY(launch_transpose(ctx->stream, Y, ctx->y.as<float>(), R, n));
    for (int k = k_begin; k < k_end; ++k) {
        VQ_TRY(stream_step(ctx, R, cur, nxt, ctx->y.as<float>(), at, k, p.dt, p.a0, p.c0,
                           k == k_end - 1 && F_last ? ctx->f.as<float>() : nullptr, rule_of(p)));
        std::swap(cur, nxt);
    }
    VQ_TRY(launch_transpose(ctx->stream, cur, S, n, R));
    VQ_TRY(launch_transpose(ctx->stream, ctx->y.as<float>(), Y, n, R));
    if (F_last) VQ_TRY(launch_transpose(ctx->stream, ctx->f.as<float>(), F_last, n, R));
    return VELOXQ_OK;
}

int veloxq_selftest_timeout(int64_t budget_cycles) {
    if (budget_cycles < 1000 || budget_cycles > 10000000000LL)
        return fail(VELOXQ_EINVAL, "budget_cycles must be in [1e3, 1e10]");
    int code = 0;
    VQ_TRY(tc_wait_selftest((long long)budget_cycles, &code));
    if (code == 0) return fail(VELOXQ_ECUDA, "the self-test wait completed although nothing arrived");
    return fail(VELOXQ_ETIMEDOUT, "bounded device wait gave up as intended (code " + std::to_string(code) + ")");
}

int veloxq_grad(veloxq_ctx* ctx, int32_t replicas, int32_t steps, const veloxq_schedule* sched, uint64_t seed,
                int32_t ckpt_every, double* loss, double* d_dt, double* d_kappa, double* d_knots) {
    if (!ctx) return fail(VELOXQ_EINVAL, "ctx must not be NULL");
    VQ_TRY(check_device(ctx));
    if (replicas < 1 || replicas > kMaxReplicas || steps < 1)
        return fail(VELOXQ_EINVAL, "replicas must be in [1, 2^20] and steps >= 1");
    if (ckpt_every < 1) return fail(VELOXQ_EINVAL, "ckpt_every must be >= 1");
    RunParams p;
    VQ_TRY(resolve(ctx, sched, steps, &p));
    if (ctx->dense || !ctx->has_csr)
        return fail(VELOXQ_EUNSUPPORTED, "the adjoint kernels run on sparse (CSR) contexts");
    if (p.method != VELOXQ_METHOD_BSB) return fail(VELOXQ_EUNSUPPORTED, "the adjoint is of the ballistic-SB step");
    const int nk = (int)p.knots.size();
    if (nk > 64) return fail(VELOXQ_EINVAL, "at most 64 schedule knots");
    CtxExtra* ex = extra(ctx);
    cudaStream_t user = ctx->stream;
    if (user == nullptr) {
        VQ_CUDA(cudaEventRecord(ex->ev, user));
        VQ_CUDA(cudaStreamWaitEvent(ex->work, ex->ev, 0));
        ctx->stream = ex->work;
    }
    struct Restore {
        veloxq_ctx* c;
        cudaStream_t s;
        ~Restore() { c->stream = s; }
    } restore{ctx, user};
    VQ_TRY(upload_schedule(ctx, p));
    const std::vector<float> a_host = schedule_table(p);
    {
        const size_t blk = sizeof(float) * (size_t)(ctx->n * (int64_t)replicas);
        DevBuf t;
        VQ_TRY(t.ensure(3 * blk));
        VQ_TRY(stream_autotune(ctx, replicas, t.as<float>(), t.as<float>() + ctx->n * (int64_t)replicas,
                               t.as<float>() + 2 * ctx->n * (int64_t)replicas));
    }
    double dc0 = 0.0;
    AdjTiming tm;
    VQ_TRY(adjoint_run(ctx, replicas, p, a_host, seed, ckpt_every, loss, d_dt, &dc0, d_knots, nk, &tm));
    ex->timing.ms_total = tm.ms_total;
    ex->timing.ms_main = tm.ms_reverse;
    ex->timing.launches = tm.launches;
    ex->timing.path = VELOXQ_PATH_STREAM;
    ex->timing.main_launches = tm.reverse_launches;
    ex->timing.stream_gather = 0;
    ex->timing.stream_chunk = 0;
    ex->timing.batch_stages = 0;
    ex->timing.batch_group = 0;
    ex->timed = true;
    if (d_kappa) {
        // c0 = kappa / rho(J) = 2 kappa / rho(Qoff) unless c0 was given
        const bool given = sched && sched->c0 > 0;
        *d_kappa = given ? dc0 : (ctx->rho > 1e-12 ? dc0 * 2.0 / ctx->rho : dc0);
    }
    return VELOXQ_OK;
}

}  // extern "C"
