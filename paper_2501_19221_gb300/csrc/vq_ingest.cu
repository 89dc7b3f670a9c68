// vq_ingest.cu -- building a context on the device: validation, the symmetric
// off-diagonal operand Qoff, the bias b, the constant K0, fixed-point energy
// weights and the spectral radius (Lanczos, or power iteration in one CTA
// for small sparse instances).
//
// Identity used throughout (Sec. 2 eq. qubo_model with x = (1 + s)/2):
//   E(x) = s^T Qoff s / 4 + b^T s / 2 + K0,  b = Qs 1 + c,
//   K0   = sum_{i != j} Qs_ij / 4 + sum_i d_i / 2,  d_i = Q_ii + c_i,
// and, for the exact energy of a binary x,
//   E(x) = sum_i x_i (d_i + sum_{j != i} Qs_ij x_j).
// Energies are accumulated as int64 multiples of 2^-S (S = energy_shift):
// exact for integer Q (S = 1, dense and sparse alike: 2 Qs is an integer)
// and, for real Q, exact sums of values rounded to 2^-S with S chosen so that
// no sum can overflow -- order-independent, unlike FP64 summation.
#include <cub/cub.cuh>

#include <cmath>
#include <cstring>

#include "vq_internal.cuh"

namespace vq {

namespace {

constexpr int kRedBlocks = 304;   // grid-stride; a fixed count fixes the order of the FP64 partial sums
constexpr int64_t kDenseCsrMax = 512;   // dense instances up to this size also keep CSR rows
constexpr int kRedThreads = 512;

template <typename T> __device__ __forceinline__ double to_d(T v) { return (double)v; }

// deterministic two-stage sum (fixed partition and tree order)
__global__ void k_sum_stage1(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
    __shared__ double sh[kRedThreads];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += x[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_stage2(const double* __restrict__ part, int nparts, double* __restrict__ out) {
    __shared__ double sh[kRedThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

int reduce_sum(cudaStream_t st, const double* x, int64_t n, double* out, double* part) {
    k_sum_stage1<<<kRedBlocks, kRedThreads, 0, st>>>(x, n, part);
    k_sum_stage2<<<1, kRedThreads, 0, st>>>(part, kRedBlocks, out);
    VQ_LAUNCH_CHECK("reduce_sum");
    return VELOXQ_OK;
}

// error word layout: bit flags, plus first offending row
enum { ERR_ROWPTR = 1, ERR_COL = 2, ERR_ORDER = 4, ERR_NONFINITE = 8, ERR_ASYM = 16, ERR_DIAG = 32,
       ERR_RANGE = 64 };

template <typename T> __device__ __forceinline__ bool finite_val(T v) { return true; }
template <> __device__ __forceinline__ bool finite_val<float>(float v) { return isfinite(v); }
template <> __device__ __forceinline__ bool finite_val<double>(double v) { return isfinite(v); }

// ------------------------------- dense ------------------------------------
template <typename T>
__global__ void k_dense_check(const T* __restrict__ q, int64_t total, int* err) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x)
        if (!finite_val(q[p])) atomicOr(err, ERR_NONFINITE);
}

// Ising: mirror the strict upper triangle into the lower one (in place).
template <typename T>
__global__ void k_dense_mirror(T* q, int64_t n) {
    const int64_t total = n * n;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = p / n, j = p % n;
        if (i > j) q[p] = q[j * n + i];
        else if (i == j) q[p] = T(0);
    }
}

// Per row: off-diagonal row sum, |.| row sum, diagonal (one block per row,
// rows row0, row0 + 1, ...).
template <typename T>
__global__ void k_dense_rows(const T* __restrict__ q, int64_t n, int64_t row0, double* rowsum, double* absrow,
                             double* diag) {
    __shared__ double s1[256], s2[256];
    const int64_t i = row0 + blockIdx.x;
    const T* row = q + i * n;
    double a = 0.0, b = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
        if (j != i) {
            const double v = to_d(row[j]);
            a += v;
            b += fabs(v);
        }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            s1[threadIdx.x] += s1[threadIdx.x + s];
            s2[threadIdx.x] += s2[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        rowsum[i] = s1[0];
        absrow[i] = s2[0];
        diag[i] = to_d(row[i]);
    }
}

// Per column: off-diagonal column sums, as partial sums over chunks of
// kColRows rows (grid: column blocks x row chunks chunk0, chunk0 + 1, ...,
// loads coalesced over the columns), then the chunks added in order for each
// column.
constexpr int kColRows = 256;
template <typename T>
__global__ void k_dense_cols_part(const T* __restrict__ q, int64_t n, int64_t chunk0, double* __restrict__ part) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t c = chunk0 + blockIdx.y;
    const int64_t i0 = c * kColRows, i1 = i0 + kColRows < n ? i0 + kColRows : n;
    if (j >= n) return;
    double a = 0.0;
#pragma unroll 8
    for (int64_t i = i0; i < i1; ++i)
        if (i != j) a += to_d(q[i * n + j]);
    part[c * n + j] = a;
}
__global__ void k_dense_cols_sum(int64_t n, int chunks, const double* __restrict__ part, double* colsum) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double a = 0.0;
    for (int c = 0; c < chunks; ++c) a += part[(int64_t)c * n + j];
    colsum[j] = a;
}

// Qoff_ij = (Q_ij + Q_ji)/2 off the diagonal, 0 on it; 32x32 tiles through
// shared memory. The sum is formed in double and rounded once to float; for
// float input the float sum scaled by 1/2 is the same value (a power-of-two
// scaling commutes with the rounding), so that case stays in float.
template <typename T> struct QoffAcc { using type = double; };
template <> struct QoffAcc<float> { using type = float; };
template <typename T>
__global__ void k_dense_qoff(const T* __restrict__ q, int64_t n, float* __restrict__ out) {
    using A = typename QoffAcc<T>::type;
    __shared__ A tile[32][33];
    const int64_t bi = (int64_t)blockIdx.y * 32, bj = (int64_t)blockIdx.x * 32;
    // load the transposed tile Q[bj.., bi..]
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t gi = bj + r, gj = bi + threadIdx.x;
        tile[r][threadIdx.x] = (gi < n && gj < n) ? (A)to_d(q[gi * n + gj]) : (A)0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t gi = bi + r, gj = bj + threadIdx.x;
        if (gi < n && gj < n) {
            const A v = (A)0.5 * ((A)to_d(q[gi * n + gj]) + tile[threadIdx.x][r]);
            out[gi * n + gj] = (gi == gj) ? 0.0f : (float)v;
        }
    }
}

// Rows of Qoff of a small dense instance as CSR (every off-diagonal entry):
// wf = Qoff_ij (field operand), wfix = round((Q_ij + Q_ji)/2 2^S) (real energies).
template <typename T>
__global__ void k_dense_to_csr(const T* __restrict__ q, int64_t n, const float* __restrict__ qoff, int shift,
                               int64_t* rp, int32_t* col, float* wf, int64_t* wfix, unsigned long long* maxw2) {
    const int64_t i = blockIdx.x;
    if (threadIdx.x == 0) {
        rp[i] = i * (n - 1);
        if (i == n - 1) rp[n] = n * (n - 1);
    }
    const double scale = ldexp(1.0, shift);
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        if (j == i) continue;
        const int64_t o = i * (n - 1) + (j < i ? j : j - 1);
        col[o] = (int32_t)j;
        wf[o] = qoff[i * n + j];
        const double w2 = to_d(q[i * n + j]) + to_d(q[j * n + i]);
        if (wfix) wfix[o] = __double2ll_rn(0.5 * w2 * scale);
        else atomicMax(maxw2, (unsigned long long)fabs(w2));
    }
}

// d_i, b_i, |d_i| for dense contexts
__global__ void k_dense_bias(int64_t n, int ising, const double* __restrict__ rowsum, const double* __restrict__ colsum,
                             const double* __restrict__ diag, const double* __restrict__ lin, double* d, float* bf,
                             double* absd) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c = lin ? lin[i] : 0.0;
    const double di = ising ? c - rowsum[i] : diag[i] + c;   // Ising: Q_ii = h_i - sum_l J_il
    d[i] = di;
    absd[i] = fabs(di);
    bf[i] = (float)(di + 0.5 * (rowsum[i] + colsum[i]));
}

// -------------------------------- CSR -------------------------------------
template <typename T>
__global__ void k_csr_validate(int64_t n, int64_t nnz, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const T* __restrict__ val, int ising, int* err, int64_t* bad_row) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t b = rp[i], e = rp[i + 1];
    int f = 0;
    // offsets are checked against the arrays before any entry is read
    if (b < 0 || e < b || e > nnz) f |= ERR_ROWPTR;
    else {
        int32_t prev = -1;
        for (int64_t p = b; p < e; ++p) {
            const int32_t j = col[p];
            if (j < 0 || (int64_t)j >= n) { f |= ERR_COL; break; }
            if (j <= prev) { f |= ERR_ORDER; break; }
            prev = j;
            if (!finite_val(val[p])) f |= ERR_NONFINITE;
            if (ising && j == i) f |= ERR_DIAG;
        }
    }
    if (f) {
        atomicOr(err, f);
        atomicMin((unsigned long long*)bad_row, (unsigned long long)i);
    }
}

__device__ __forceinline__ int64_t find_in_row(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                               int64_t row, int32_t target) {
    int64_t lo = rp[row], hi = rp[row + 1] - 1;
    while (lo <= hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int32_t c = col[mid];
        if (c == target) return mid;
        if (c < target) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// Symmetric value of the stored entry p = (i, j), i != j.
template <typename T>
__device__ __forceinline__ bool sym_value(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                          const T* __restrict__ val, int64_t i, int64_t p, int ising,
                                          double* qs, int64_t* w2) {
    const int32_t j = col[p];
    const int64_t t = find_in_row(rp, col, j, (int32_t)i);
    if (t < 0) return false;
    const double vij = to_d(val[p]), vji = to_d(val[t]);
    if (ising) {
        // the pair's coupling is the value stored at its upper-triangle position
        const double v = (i < j) ? vij : vji;
        *qs = v;
        *w2 = (int64_t)(2.0 * v);
    } else {
        *qs = 0.5 * (vij + vji);
        *w2 = (int64_t)vij + (int64_t)vji;
    }
    return true;
}

template <typename T>
__global__ void k_csr_pass1(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const T* __restrict__ val, int ising, int integer, int64_t* cnt, double* rowsum,
                            double* absrow, double* diag, int* err, int64_t* bad_row, unsigned long long* maxw2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t c = 0;
    double rs = 0.0, ab = 0.0, dg = 0.0;
    unsigned long long mw = 0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        if ((int64_t)col[p] == i) { dg = to_d(val[p]); continue; }
        double qs;
        int64_t w2;
        if (!sym_value(rp, col, val, i, p, ising, &qs, &w2)) {
            atomicOr(err, ERR_ASYM);
            atomicMin((unsigned long long*)bad_row, (unsigned long long)i);
            return;
        }
        ++c;
        rs += qs;
        ab += fabs(qs);
        if (integer) {
            const unsigned long long a = (unsigned long long)(w2 < 0 ? -w2 : w2);
            if (a > mw) mw = a;
        }
    }
    cnt[i] = c;
    rowsum[i] = rs;
    absrow[i] = ab;
    diag[i] = dg;
    if (integer && mw) atomicMax(maxw2, mw);
}

template <typename T>
__global__ void k_csr_pass2(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const T* __restrict__ val, int ising, int integer, int shift,
                            const int64_t* __restrict__ rp_f, int32_t* col_f, float* wf, int8_t* w8, int64_t* wfix) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t o = rp_f[i];
    const double scale = ldexp(1.0, shift);
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        if ((int64_t)col[p] == i) continue;
        double qs;
        int64_t w2;
        sym_value(rp, col, val, i, p, ising, &qs, &w2);
        col_f[o] = col[p];
        wf[o] = (float)qs;
        if (w8) w8[o] = (int8_t)w2;
        if (wfix) wfix[o] = integer ? w2 : __double2ll_rn(qs * scale);
        ++o;
    }
}

__global__ void k_csr_bias(int64_t n, int ising, const double* __restrict__ rowsum, const double* __restrict__ diag,
                           const double* __restrict__ lin, double* d, float* bf, double* absd) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c = lin ? lin[i] : 0.0;
    const double di = ising ? c - rowsum[i] : diag[i] + c;
    d[i] = di;
    absd[i] = fabs(di);
    bf[i] = (float)(di + rowsum[i]);
}

__global__ void k_fix(int64_t n, const double* __restrict__ d, int shift, int64_t* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = __double2ll_rn(d[i] * ldexp(1.0, shift));
}

// ------------------------- spectral radius of Qoff -------------------------
// FP32 vectors and products (FP64 runs at a small fraction of the FP32 rate
// on this part, and the estimate only scales c0); sums over blocks in FP64 in
// a fixed order. pi_start is the fixed, seed-free start vector of both
// estimates below: entries of magnitude in [1, 1.25) with hashed signs.
__device__ __forceinline__ float pi_start(int64_t i) {
    uint32_t h = (uint32_t)i * 2654435761u;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    const float mag = 1.0f + (float)((h >> 1) & 1023u) / 4096.0f;
    return (h & 1u) ? mag : -mag;
}
__device__ __forceinline__ float warp_sum_to_lane0(float a) {
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    return a;
}
constexpr int kPiBlock = 256;

// ---- Lanczos estimate of rho(Qoff) (dense, and sparse beyond one CTA) ------
// Plain Lanczos from the fixed start vector pi_start: m steps
//   u = A v_j, alpha_j = v_j . u, w_{j+1} = u - alpha_j v_j - beta_j v_{j-1},
//   beta_{j+1} = |w_{j+1}|, v_{j+1} = w_{j+1} / beta_{j+1},
// and rho ~ max |extreme eigenvalue| of the m x m tridiagonal T (alpha on the
// diagonal, beta beside it). Ritz values lie inside the spectrum, so the
// estimate approaches rho from below, far faster than the power iteration for
// the continuous spectra of these instances (dense Gaussian, Wishart,
// lattices: within 2 % of rho after the 32 steps taken). The vectors are stored
// unnormalised (w_j, with |w_j|^2 kept in FP64), so that each step is one
// matrix pass and one vector pass; products are FP32, every sum over blocks
// FP64 in a fixed order. No reorthogonalisation: the loss of orthogonality
// repeats converged Ritz values but does not move the extreme ones.
constexpr int kLzSteps = 32;
struct LzScal {
    double* part;      // one partial per block
    unsigned* count;   // blocks finished in this launch (reset by the last one)
    double* alpha;     // [kLzSteps]      alpha_j
    double* nrm2;      // [kLzSteps + 1]  |w_j|^2
};
__device__ __forceinline__ float inv_norm(double q) { return q > 0.0 ? (float)(1.0 / sqrt(q)) : 0.0f; }
// Called by every thread of the block with its own partial; the last block
// to finish writes the total over blocks (FP64, fixed order) to *out.
__device__ __forceinline__ void lz_block_finish(float v, LzScal sc, double* out) {
    __shared__ float wsum[kPiBlock / 32];
    __shared__ double dsum[kPiBlock];
    __shared__ bool last;
    v = warp_sum_to_lane0(v);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.0f;
        for (int q = 0; q < kPiBlock / 32; ++q) b += wsum[q];
        sc.part[blockIdx.x] = (double)b;
        __threadfence();
        last = atomicAdd(sc.count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    double a = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += kPiBlock) a += __ldcg(sc.part + i);
    dsum[threadIdx.x] = a;
    __syncthreads();
    for (int s = kPiBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) dsum[threadIdx.x] += dsum[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *out = dsum[0];
        *sc.count = 0u;
    }
}
// w_0 = the fixed start vector; |w_0|^2
__global__ void __launch_bounds__(kPiBlock) k_lz_start(int64_t n, float* __restrict__ w, LzScal sc) {
    float sq = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * kPiBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kPiBlock) {
        const float x = pi_start(i);
        w[i] = x;
        sq = fmaf(x, x, sq);
    }
    lz_block_finish(sq, sc, sc.nrm2);
}
// u = A v_j (v_j = w_j / |w_j|) for CSR rows, and alpha_j = v_j . u; odd
// steps walk the rows backwards so that the ones the previous pass read last
// (still in L2) come first.
__global__ void __launch_bounds__(kPiBlock) k_lz_spmv(int64_t n, const int64_t* __restrict__ rp,
                                                     const int32_t* __restrict__ col, const float* __restrict__ wf,
                                                     const float* __restrict__ wj, float* __restrict__ u, LzScal sc,
                                                     int j) {
    const float inv = inv_norm(sc.nrm2[j]);
    const bool rev = j & 1;
    float dot = 0.0f;
    for (int64_t k = (int64_t)blockIdx.x * kPiBlock + threadIdx.x; k < n; k += (int64_t)gridDim.x * kPiBlock) {
        const int64_t i = rev ? n - 1 - k : k;
        float a = 0.0f;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) a = fmaf(wf[p], wj[col[p]], a);
        a *= inv;
        u[i] = a;
        dot = fmaf(a, wj[i] * inv, dot);
    }
    lz_block_finish(dot, sc, sc.alpha + j);
}
// The same for a dense Qoff: one warp per row, 16-byte loads when n % 4 == 0.
__global__ void __launch_bounds__(kPiBlock) k_lz_gemv(int64_t n, const float* __restrict__ q,
                                                     const float* __restrict__ wj, float* __restrict__ u, LzScal sc,
                                                     int j) {
    const float inv = inv_norm(sc.nrm2[j]);
    const bool rev = j & 1;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (kPiBlock / 32);
    float dot = 0.0f;
    for (int64_t k = (int64_t)blockIdx.x * (kPiBlock / 32) + (threadIdx.x >> 5); k < n; k += nwarps) {
        const int64_t i = rev ? n - 1 - k : k;
        const float* row = q + i * n;
        float a = 0.0f;
        if ((n & 3) == 0) {
            const float4* r4 = reinterpret_cast<const float4*>(row);
            const float4* v4 = reinterpret_cast<const float4*>(wj);
            // eight 16-byte loads per lane in flight, summed in a fixed order
            const int64_t n4 = n / 4;
            int64_t c = lane;
            for (; c + 7 * 32 < n4; c += 8 * 32) {
                float4 x[8], y[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    x[u] = __ldcs(r4 + c + u * 32);
                    y[u] = v4[c + u * 32];
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    a = fmaf(x[u].x, y[u].x, a);
                    a = fmaf(x[u].y, y[u].y, a);
                    a = fmaf(x[u].z, y[u].z, a);
                    a = fmaf(x[u].w, y[u].w, a);
                }
            }
            for (; c < n4; c += 32) {
                const float4 x = __ldcs(r4 + c), y = v4[c];
                a = fmaf(x.x, y.x, a);
                a = fmaf(x.y, y.y, a);
                a = fmaf(x.z, y.z, a);
                a = fmaf(x.w, y.w, a);
            }
        } else {
            for (int64_t c = lane; c < n; c += 32) a = fmaf(row[c], wj[c], a);
        }
        a = warp_sum_to_lane0(a);
        if (lane == 0) {
            a *= inv;
            u[i] = a;
            dot = fmaf(a, wj[i] * inv, dot);
        }
    }
    lz_block_finish(dot, sc, sc.alpha + j);
}
// w_{j+1} = u - alpha_j v_j - beta_j v_{j-1} in place of u, and |w_{j+1}|^2
// (beta_j = |w_j|, v_j = w_j / |w_j|).
__global__ void __launch_bounds__(kPiBlock) k_lz_update(int64_t n, float* __restrict__ u, const float* __restrict__ wj,
                                                       const float* __restrict__ wjm1, LzScal sc, int j) {
    const double nj = sc.nrm2[j];
    const float c1 = (float)(sc.alpha[j] * (nj > 0.0 ? 1.0 / sqrt(nj) : 0.0));
    const float c2 = (j > 0 && sc.nrm2[j - 1] > 0.0) ? (float)sqrt(nj / sc.nrm2[j - 1]) : 0.0f;
    float sq = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * kPiBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kPiBlock) {
        float w = fmaf(-c1, wj[i], u[i]);
        if (j > 0) w = fmaf(-c2, wjm1[i], w);
        u[i] = w;
        sq = fmaf(w, w, sq);
    }
    lz_block_finish(sq, sc, sc.nrm2 + j + 1);
}

// Extreme eigenvalues of the symmetric tridiagonal matrix (diagonal a[0..m),
// off-diagonal b[0..m-1)) by bisection on the Sturm count (the number of
// negative pivots of T - x I counts the eigenvalues below x).
int sturm_below(const std::vector<double>& a, const std::vector<double>& b, double x) {
    int c = 0;
    double d = 1.0;
    for (size_t i = 0; i < a.size(); ++i) {
        const double off = i ? b[i - 1] * b[i - 1] : 0.0;
        d = a[i] - x - (i ? off / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++c;
    }
    return c;
}
void tridiag_extremes(const std::vector<double>& a, const std::vector<double>& b, double* lo, double* hi) {
    double g0 = a[0], g1 = a[0];
    for (size_t i = 0; i < a.size(); ++i) {
        const double r = (i ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < a.size() ? std::fabs(b[i]) : 0.0);
        g0 = std::min(g0, a[i] - r);
        g1 = std::max(g1, a[i] + r);
    }
    const int m = (int)a.size();
    double l = g0, h = g1;   // smallest eigenvalue: largest x with no eigenvalue below
    for (int it = 0; it < 200 && h - l > 1e-15 * std::max(1.0, std::fabs(l) + std::fabs(h)); ++it) {
        const double x = 0.5 * (l + h);
        if (sturm_below(a, b, x) >= 1) h = x; else l = x;
    }
    *lo = 0.5 * (l + h);
    l = g0;
    h = g1;                  // largest eigenvalue: smallest x with every eigenvalue below
    for (int it = 0; it < 200 && h - l > 1e-15 * std::max(1.0, std::fabs(l) + std::fabs(h)); ++it) {
        const double x = 0.5 * (l + h);
        if (sturm_below(a, b, x) >= m) h = x; else l = x;
    }
    *hi = 0.5 * (l + h);
}

// Power iteration for a small sparse instance in ONE CTA (no launch per
// iteration): v, w and the rows in shared memory, FP32 arithmetic. With
// W > 0 the rows are stored as W slots each, slot-major (slot k of row i at
// k n + i), short rows padded with zero weights on their own column, and the
// slot loop is unrolled; W = 0 keeps the CSR rows. Either way a row is summed
// in CSR order. Each thread sums the squares of the rows it writes; one
// barrier per iteration publishes both w and the per-warp partials, which
// every warp then reduces in the same fixed order, so all threads hold the
// same 1/|w|. The partials alternate between two arrays: the next write to
// one of them comes after the following barrier, when every warp has read it.
constexpr int kPiThreads = 1024;
constexpr int kPiWarps = kPiThreads / 32;
constexpr int64_t kPiSingleMaxN = 8192;
constexpr size_t kPiSmemMax = 200 * 1024;
__host__ __device__ inline size_t pi_smem(int64_t n, int64_t nnz, int W) {
    if (W > 0) return sizeof(float) * 2 * (size_t)n + (sizeof(int32_t) + sizeof(float)) * (size_t)n * (size_t)W;
    return sizeof(float) * 2 * (size_t)n + sizeof(int32_t) * (size_t)(n + 1) +
           (sizeof(int32_t) + sizeof(float)) * (size_t)nnz;
}
template <int W>
__global__ void __launch_bounds__(kPiThreads) k_pi_single(int32_t n, int32_t nnz, int iters,
                                                          const int64_t* __restrict__ rp_g,
                                                          const int32_t* __restrict__ col_g,
                                                          const float* __restrict__ wq_g, double* out) {
    extern __shared__ __align__(16) unsigned char pis_raw[];
    float* v = reinterpret_cast<float*>(pis_raw);
    float* w = v + n;
    int32_t* rp = reinterpret_cast<int32_t*>(w + n);                       // W = 0
    int32_t* col = W > 0 ? reinterpret_cast<int32_t*>(w + n) : rp + (n + 1);
    float* wq = reinterpret_cast<float*>(col + (W > 0 ? W * n : nnz));
    __shared__ float red[2][kPiWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // |x|^2 from the per-warp partials of one array, identical in every thread
    auto all_norm2 = [&](const float* part) {
        return __shfl_sync(0xffffffffu, warp_sum_to_lane0(part[lane]), 0);
    };
    if constexpr (W > 0) {
        for (int i = threadIdx.x; i < n; i += kPiThreads) {
            const int p0 = (int)rp_g[i], deg = (int)(rp_g[i + 1] - rp_g[i]);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                col[k * n + i] = k < deg ? col_g[p0 + k] : i;
                wq[k * n + i] = k < deg ? wq_g[p0 + k] : 0.0f;
            }
        }
    } else {
        for (int i = threadIdx.x; i <= n; i += kPiThreads) rp[i] = (int32_t)rp_g[i];
        for (int p = threadIdx.x; p < nnz; p += kPiThreads) {
            col[p] = col_g[p];
            wq[p] = wq_g[p];
        }
    }
    // (Qoff v)_i in CSR order
    auto row_dot = [&](const float* x, int i) {
        float a = 0.0f;
        if constexpr (W > 0) {
#pragma unroll
            for (int k = 0; k < W; ++k) a = fmaf(wq[k * n + i], x[col[k * n + i]], a);
        } else {
            for (int p = rp[i]; p < rp[i + 1]; ++p) a = fmaf(wq[p], x[col[p]], a);
        }
        return a;
    };
    float sq = 0.0f;
    for (int i = threadIdx.x; i < n; i += kPiThreads) {
        const float x = pi_start(i);
        v[i] = x;
        sq = fmaf(x, x, sq);
    }
    sq = warp_sum_to_lane0(sq);
    if (lane == 0) red[0][warp] = sq;
    __syncthreads();
    float nrm2 = all_norm2(red[0]);
    for (int t = 0; t < iters; ++t) {
        const float inv = nrm2 > 0.0f ? 1.0f / sqrtf(nrm2) : 0.0f;
        float* part = red[(t + 1) & 1];
        sq = 0.0f;
        // two rows at a time (the second clamped into range, kept only when
        // it exists) so that both rows' loads are in flight together
        for (int i0 = threadIdx.x; i0 < n; i0 += 2 * kPiThreads) {
            const int i1 = i0 + kPiThreads;
            const float a0 = row_dot(v, i0) * inv;
            const float a1 = row_dot(v, i1 < n ? i1 : i0) * inv;
            w[i0] = a0;
            sq = fmaf(a0, a0, sq);
            if (i1 < n) {
                w[i1] = a1;
                sq = fmaf(a1, a1, sq);
            }
        }
        sq = warp_sum_to_lane0(sq);
        if (lane == 0) part[warp] = sq;
        __syncthreads();
        nrm2 = all_norm2(part);
        float* tmp = v;
        v = w;
        w = tmp;
    }
    if (threadIdx.x == 0) *out = (double)nrm2;
}

template <typename T>
int ingest_dense_t(veloxq_ctx* ctx, const void* Qh, const double* ch, bool ising, bool integer) {
    const int64_t n = ctx->n;
    cudaStream_t st = ctx->stream;
    const size_t qbytes = sizeof(T) * (size_t)n * (size_t)n;
    VQ_TRY(ctx->qx.ensure(qbytes));
    T* q = ctx->qx.as<T>();
    DevBuf tmp;
    // rowsum, colsum, absrow, diag, lin, d, absd, part, scalars, column-sum chunks
    const int col_chunks = (int)div_up(n, kColRows);
    VQ_TRY(tmp.ensure(sizeof(double) * (size_t)(7 * n + kRedBlocks + 16 + (int64_t)col_chunks * n) + 64));
    double* rowsum = tmp.as<double>();
    double* colsum = rowsum + n;
    double* absrow = colsum + n;
    double* diag = absrow + n;
    double* lin = diag + n;
    double* d = lin + n;
    double* absd = d + n;
    double* part = absd + n;
    double* scal = part + kRedBlocks;          // [0] sum rowsum [1] sum d [2] sum absrow [3] sum absd [4] sum lin
    int* err = (int*)(scal + 8);
    double* cpart = scal + 8 + 8;              // [col_chunks][n]
    VQ_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    if (ch) VQ_CUDA(cudaMemcpyAsync(lin, ch, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    else VQ_CUDA(cudaMemsetAsync(lin, 0, sizeof(double) * n, st));
    const int64_t total = n * n;
    const int gb = (int)std::min<int64_t>(div_up(total, 256), (int64_t)device_sms(ctx->device) * 16);
    // Q goes up in row chunks (whole kColRows blocks) on a helper stream; the
    // checks, row sums and column partial sums of a chunk run on the context
    // stream as soon as it has arrived, under the upload of the next one. The
    // sums are the same as over the whole matrix at once (per row, and per
    // kColRows-row chunk of a column). Ising input is mirrored across the
    // diagonal first, which needs every row: it goes up in one piece.
    const int64_t rows_per = (ising || n < 4 * kColRows) ? n : div_up(div_up(n, 4), kColRows) * kColRows;
    const int nup = (int)div_up(n, rows_per);
    struct Upload {
        cudaStream_t s = nullptr;
        std::vector<cudaEvent_t> ev;
        ~Upload() {
            for (cudaEvent_t e : ev)
                if (e) cudaEventDestroy(e);
            if (s) cudaStreamDestroy(s);   // released once its copies are done
        }
    } up;
    if (nup > 1) {
        VQ_CUDA(cudaStreamCreateWithFlags(&up.s, cudaStreamNonBlocking));
        up.ev.assign((size_t)nup + 1, nullptr);
        for (cudaEvent_t& e : up.ev) VQ_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        VQ_CUDA(cudaEventRecord(up.ev[0], st));            // after everything enqueued on the context stream
        VQ_CUDA(cudaStreamWaitEvent(up.s, up.ev[0], 0));
    }
    const T* Qt = static_cast<const T*>(Qh);
    for (int c = 0; c < nup; ++c) {
        const int64_t r0 = c * rows_per, r1 = std::min<int64_t>(n, r0 + rows_per);
        const int64_t cnt = (r1 - r0) * n;
        if (nup > 1) {
            VQ_CUDA(cudaMemcpyAsync(q + r0 * n, Qt + r0 * n, sizeof(T) * (size_t)cnt, cudaMemcpyHostToDevice, up.s));
            VQ_CUDA(cudaEventRecord(up.ev[(size_t)c + 1], up.s));
            VQ_CUDA(cudaStreamWaitEvent(st, up.ev[(size_t)c + 1], 0));
        } else {
            VQ_CUDA(cudaMemcpyAsync(q, Qh, qbytes, cudaMemcpyHostToDevice, st));
        }
        const int gbc = (int)std::min<int64_t>(div_up(cnt, 256), (int64_t)gb);
        k_dense_check<T><<<gbc, 256, 0, st>>>(q + r0 * n, cnt, err);
        if (ising) k_dense_mirror<T><<<gb, 256, 0, st>>>(q, n);
        k_dense_rows<T><<<(unsigned)(r1 - r0), 256, 0, st>>>(q, n, r0, rowsum, absrow, diag);
        k_dense_cols_part<T><<<dim3((unsigned)div_up(n, 128), (unsigned)div_up(r1 - r0, kColRows)), 128, 0, st>>>(
            q, n, r0 / kColRows, cpart);
    }
    k_dense_cols_sum<<<(unsigned)div_up(n, 256), 256, 0, st>>>(n, col_chunks, cpart, colsum);
    VQ_TRY(ctx->qoff32.ensure(sizeof(float) * (size_t)total));
    dim3 tb(32, 8), tg((unsigned)div_up(n, 32), (unsigned)div_up(n, 32));
    k_dense_qoff<T><<<tg, tb, 0, st>>>(q, n, ctx->qoff32.as<float>());
    VQ_TRY(ctx->bf.ensure(sizeof(float) * n));
    k_dense_bias<<<(unsigned)div_up(n, 256), 256, 0, st>>>(n, ising ? 1 : 0, rowsum, colsum, diag,
                                                            lin, d, ctx->bf.as<float>(), absd);
    VQ_LAUNCH_CHECK("dense ingest");
    VQ_TRY(reduce_sum(st, rowsum, n, scal + 0, part));
    VQ_TRY(reduce_sum(st, d, n, scal + 1, part));
    VQ_TRY(reduce_sum(st, absrow, n, scal + 2, part));
    VQ_TRY(reduce_sum(st, absd, n, scal + 3, part));
    VQ_TRY(reduce_sum(st, lin, n, scal + 4, part));
    double hs[5];
    int herr = 0;
    VQ_CUDA(cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, st));
    VQ_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    VQ_CUDA(cudaStreamSynchronize(st));
    if (herr & ERR_NONFINITE) return fail(VELOXQ_EINVAL, "coupling matrix holds a non-finite value");
    ctx->K0 = 0.25 * hs[0] + 0.5 * hs[1];
    ctx->ising_offset = ising ? 0.5 * hs[0] - hs[4] : 0.0;
    const double Tsum = hs[2] + hs[3];
    if (integer) {
        if (Tsum >= 4.0e18) return fail(VELOXQ_EUNSUPPORTED, "integer couplings too large for int64 energies");
        ctx->energy_shift = 1;            // energies held as 2E, like sparse contexts (2 Qs is an integer)
    } else {
        int e = 0;
        std::frexp(Tsum > 0 ? Tsum : 1.0, &e);     // Tsum < 2^e
        // every fixed-point sum stays below 2^62 only while Tsum < 2^61
        if (61 - e < 0) return fail(VELOXQ_EUNSUPPORTED, "real couplings too large for exact fixed-point energies "
                                                         "(sum |Q| + sum |c| must be below 2^61)");
        ctx->energy_shift = std::min(200, 61 - e);
    }
    VQ_TRY(ctx->dfix.ensure(sizeof(int64_t) * n));
    k_fix<<<(unsigned)div_up(n, 256), 256, 0, st>>>(n, d, ctx->energy_shift, ctx->dfix.as<int64_t>());
    VQ_LAUNCH_CHECK("dense ingest fix");
    VQ_CUDA(cudaStreamSynchronize(st));
    ctx->nnz = n * (n - 1);
    ctx->max_row = (int)(n - 1);
    if (n <= kDenseCsrMax && n > 1) {
        // small dense instances also get the rows of Qoff in CSR form so that
        // the one-launch resident kernel can run them
        const int64_t nnz = n * (n - 1);
        VQ_TRY(ctx->rowptr.ensure(sizeof(int64_t) * (n + 1)));
        VQ_TRY(ctx->col.ensure(sizeof(int32_t) * nnz));
        VQ_TRY(ctx->wf.ensure(sizeof(float) * nnz));
        if (!integer) VQ_TRY(ctx->wfix.ensure(sizeof(int64_t) * nnz));
        unsigned long long* dmax = (unsigned long long*)(scal + 6);
        VQ_CUDA(cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), st));
        k_dense_to_csr<T><<<(unsigned)n, 256, 0, st>>>(q, n, ctx->qoff32.as<float>(), ctx->energy_shift,
                                                        ctx->rowptr.as<int64_t>(), ctx->col.as<int32_t>(),
                                                        ctx->wf.as<float>(), integer ? nullptr : ctx->wfix.as<int64_t>(),
                                                        dmax);
        VQ_LAUNCH_CHECK("dense to csr");
        unsigned long long hm = 0;
        VQ_CUDA(cudaMemcpyAsync(&hm, dmax, sizeof(hm), cudaMemcpyDeviceToHost, st));
        VQ_CUDA(cudaStreamSynchronize(st));
        ctx->has_csr = true;
        ctx->wf_half_exact = integer && hm <= 2047;
    }
    return VELOXQ_OK;
}

template <typename T>
int ingest_csr_t(veloxq_ctx* ctx, const int64_t* rph, const int32_t* colh, const void* valh, const double* ch,
                 bool ising, bool integer) {
    const int64_t n = ctx->n;
    cudaStream_t st = ctx->stream;
    if (rph[0] != 0) return fail(VELOXQ_EINVAL, "rowptr[0] must be 0");
    const int64_t nnz_in = rph[n];
    if (nnz_in < 0) return fail(VELOXQ_EINVAL, "rowptr[n] must be >= 0");
    if (nnz_in > 0 && (!colh || !valh)) return fail(VELOXQ_EINVAL, "col and val must not be NULL when nnz > 0");
    DevBuf d_rp, d_col, d_val, tmp;
    VQ_TRY(d_rp.ensure(sizeof(int64_t) * (n + 1)));
    VQ_TRY(d_col.ensure(sizeof(int32_t) * std::max<int64_t>(nnz_in, 1)));
    VQ_TRY(d_val.ensure(sizeof(T) * std::max<int64_t>(nnz_in, 1)));
    VQ_CUDA(cudaMemcpyAsync(d_rp.p, rph, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
    if (nnz_in > 0) {
        VQ_CUDA(cudaMemcpyAsync(d_col.p, colh, sizeof(int32_t) * nnz_in, cudaMemcpyHostToDevice, st));
        VQ_CUDA(cudaMemcpyAsync(d_val.p, valh, sizeof(T) * nnz_in, cudaMemcpyHostToDevice, st));
    }
    // rowsum, absrow, diag, lin, d, absd | cnt (n+1) | part | scalars | err, bad_row, maxw2
    VQ_TRY(tmp.ensure(sizeof(double) * (size_t)(6 * n + (n + 1) + kRedBlocks + 8) + 256));
    double* rowsum = tmp.as<double>();
    double* absrow = rowsum + n;
    double* diag = absrow + n;
    double* lin = diag + n;
    double* d = lin + n;
    double* absd = d + n;
    int64_t* cnt = (int64_t*)(absd + n);
    double* part = (double*)(cnt + n + 1);
    double* scal = part + kRedBlocks;
    int* err = (int*)(scal + 8);
    int64_t* bad_row = (int64_t*)(scal + 9);
    unsigned long long* maxw2 = (unsigned long long*)(scal + 10);
    VQ_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    VQ_CUDA(cudaMemsetAsync(bad_row, 0x7f, sizeof(int64_t), st));
    VQ_CUDA(cudaMemsetAsync(maxw2, 0, sizeof(unsigned long long), st));
    VQ_CUDA(cudaMemsetAsync(cnt + n, 0, sizeof(int64_t), st));
    if (ch) VQ_CUDA(cudaMemcpyAsync(lin, ch, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    else VQ_CUDA(cudaMemsetAsync(lin, 0, sizeof(double) * n, st));
    const unsigned gr = (unsigned)div_up(n, 256);
    const int64_t* rp = d_rp.as<int64_t>();
    const int32_t* cl = d_col.as<int32_t>();
    const T* vl = d_val.as<T>();
    k_csr_validate<T><<<gr, 256, 0, st>>>(n, nnz_in, rp, cl, vl, ising ? 1 : 0, err, bad_row);
    int herr = 0;
    int64_t hbad = 0;
    VQ_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    VQ_CUDA(cudaMemcpyAsync(&hbad, bad_row, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    VQ_CUDA(cudaStreamSynchronize(st));
    VQ_LAUNCH_CHECK("csr validate");
    if (herr) {
        std::string m = "malformed CSR input at row " + std::to_string(hbad) + ":";
        if (herr & ERR_ROWPTR) m += " rowptr decreases or leaves [0, rowptr[n]];";
        if (herr & ERR_COL) m += " column index out of range;";
        if (herr & ERR_ORDER) m += " column indices not strictly increasing;";
        if (herr & ERR_NONFINITE) m += " non-finite value;";
        if (herr & ERR_DIAG) m += " Ising couplings must not hold diagonal entries;";
        return fail(VELOXQ_EINVAL, m);
    }
    k_csr_pass1<T><<<gr, 256, 0, st>>>(n, rp, cl, vl, ising ? 1 : 0, integer ? 1 : 0, cnt, rowsum, absrow, diag,
                                       err, bad_row, maxw2);
    VQ_LAUNCH_CHECK("csr pass1");
    unsigned long long hmaxw = 0;
    VQ_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    VQ_CUDA(cudaMemcpyAsync(&hbad, bad_row, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    VQ_CUDA(cudaMemcpyAsync(&hmaxw, maxw2, sizeof(hmaxw), cudaMemcpyDeviceToHost, st));
    VQ_CUDA(cudaStreamSynchronize(st));
    if (herr & ERR_ASYM)
        return fail(VELOXQ_EUNSUPPORTED, "CSR pattern is not structurally symmetric (row " + std::to_string(hbad) +
                                             " has an entry whose transpose is missing)");
    // exclusive scan of the per-row counts -> field rowptr
    VQ_TRY(ctx->rowptr.ensure(sizeof(int64_t) * (n + 1)));
    size_t tbytes = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tbytes, cnt, ctx->rowptr.as<int64_t>(), n + 1, st);
    DevBuf ctmp;
    VQ_TRY(ctmp.ensure(tbytes + 16));
    VQ_CUDA(cub::DeviceScan::ExclusiveSum(ctmp.p, tbytes, cnt, ctx->rowptr.as<int64_t>(), n + 1, st));
    int64_t nnz_f = 0;
    VQ_CUDA(cudaMemcpyAsync(&nnz_f, ctx->rowptr.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    VQ_TRY(ctx->bf.ensure(sizeof(float) * n));
    k_csr_bias<<<gr, 256, 0, st>>>(n, ising ? 1 : 0, rowsum, diag, lin, d, ctx->bf.as<float>(), absd);
    VQ_LAUNCH_CHECK("csr bias");
    VQ_TRY(reduce_sum(st, rowsum, n, scal + 0, part));
    VQ_TRY(reduce_sum(st, d, n, scal + 1, part));
    VQ_TRY(reduce_sum(st, absrow, n, scal + 2, part));
    VQ_TRY(reduce_sum(st, absd, n, scal + 3, part));
    VQ_TRY(reduce_sum(st, lin, n, scal + 4, part));
    double hs[5];
    VQ_CUDA(cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, st));
    VQ_CUDA(cudaStreamSynchronize(st));
    ctx->nnz = nnz_f;
    ctx->K0 = 0.25 * hs[0] + 0.5 * hs[1];
    ctx->ising_offset = ising ? 0.5 * hs[0] - hs[4] : 0.0;
    const double Tm = hs[2] + hs[3];
    if (integer) {
        if (Tm >= 4.0e18 || hmaxw > (unsigned long long)INT32_MAX)
            return fail(VELOXQ_EUNSUPPORTED, "integer couplings too large for int64 energies");
        ctx->energy_shift = 1;            // 2 Qs is an integer
    } else {
        int e = 0;
        std::frexp(Tm > 0 ? Tm : 1.0, &e);
        if (61 - e < 0) return fail(VELOXQ_EUNSUPPORTED, "real couplings too large for exact fixed-point energies "
                                                         "(sum |Q| + sum |c| must be below 2^61)");
        ctx->energy_shift = std::min(200, 61 - e);
    }
    const bool use8 = integer && hmaxw <= 127;
    ctx->wf_half_exact = integer && hmaxw <= 2047;
    VQ_TRY(ctx->col.ensure(sizeof(int32_t) * std::max<int64_t>(nnz_f, 1)));
    VQ_TRY(ctx->wf.ensure(sizeof(float) * std::max<int64_t>(nnz_f, 1)));
    if (use8) {
        VQ_TRY(ctx->w8.ensure(sizeof(int8_t) * std::max<int64_t>(nnz_f, 1) + 16));
        ctx->wfix.release();
    } else {
        VQ_TRY(ctx->wfix.ensure(sizeof(int64_t) * std::max<int64_t>(nnz_f, 1)));
        ctx->w8.release();
    }
    k_csr_pass2<T><<<gr, 256, 0, st>>>(n, rp, cl, vl, ising ? 1 : 0, integer ? 1 : 0, ctx->energy_shift,
                                       ctx->rowptr.as<int64_t>(), ctx->col.as<int32_t>(), ctx->wf.as<float>(),
                                       use8 ? ctx->w8.as<int8_t>() : nullptr,
                                       use8 ? nullptr : ctx->wfix.as<int64_t>());
    VQ_TRY(ctx->dfix.ensure(sizeof(int64_t) * n));
    k_fix<<<gr, 256, 0, st>>>(n, d, integer ? 1 : ctx->energy_shift, ctx->dfix.as<int64_t>());
    VQ_LAUNCH_CHECK("csr pass2");
    // longest row of the field structure (for kernel selection)
    {
        std::vector<int64_t> hcnt;
        // counts are small relative to the arrays; read back only their maximum
        size_t mb = 0;
        int64_t* dmax = (int64_t*)(scal + 11);
        cub::DeviceReduce::Max(nullptr, mb, cnt, dmax, n, st);
        DevBuf mtmp;
        VQ_TRY(mtmp.ensure(mb + 16));
        VQ_CUDA(cub::DeviceReduce::Max(mtmp.p, mb, cnt, dmax, n, st));
        int64_t hm = 0, hmin = 0;
        VQ_CUDA(cudaMemcpyAsync(&hm, dmax, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        int64_t* dmin = (int64_t*)(scal + 12);
        size_t nb = 0;
        cub::DeviceReduce::Min(nullptr, nb, cnt, dmin, n, st);
        DevBuf ntmp;
        VQ_TRY(ntmp.ensure(nb + 16));
        VQ_CUDA(cub::DeviceReduce::Min(ntmp.p, nb, cnt, dmin, n, st));
        VQ_CUDA(cudaMemcpyAsync(&hmin, dmin, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        VQ_CUDA(cudaStreamSynchronize(st));
        ctx->max_row = (int)hm;
        ctx->uniform_deg = (hm == hmin && hm < (1 << 20)) ? (int)hm : -1;
    }
    return VELOXQ_OK;
}

}  // namespace

int ingest_dense(veloxq_ctx* ctx, veloxq_vtype vt, const void* Qh, const double* ch, bool ising) {
    ctx->dense = true;
    ctx->qx_type = vt;
    bool integer = (vt == VELOXQ_I8 || vt == VELOXQ_I32);
    if (integer && ch)
        for (int64_t i = 0; i < ctx->n; ++i)
            if (!(std::fabs(ch[i]) < 4.0e15) || ch[i] != std::floor(ch[i])) { integer = false; break; }
    if (ch)
        for (int64_t i = 0; i < ctx->n; ++i)
            if (!std::isfinite(ch[i])) return fail(VELOXQ_EINVAL, "linear term holds a non-finite value");
    ctx->integer = integer;
    switch (vt) {
        case VELOXQ_I8: return ingest_dense_t<int8_t>(ctx, Qh, ch, ising, integer);
        case VELOXQ_I32: return ingest_dense_t<int32_t>(ctx, Qh, ch, ising, integer);
        case VELOXQ_F32: return ingest_dense_t<float>(ctx, Qh, ch, ising, integer);
        case VELOXQ_F64: return ingest_dense_t<double>(ctx, Qh, ch, ising, integer);
    }
    return fail(VELOXQ_EINVAL, "unknown value type");
}

int ingest_csr(veloxq_ctx* ctx, const int64_t* rowptr, const int32_t* col, veloxq_vtype vt, const void* val,
               const double* ch, bool ising) {
    ctx->dense = false;
    ctx->has_csr = true;
    bool integer = (vt == VELOXQ_I8 || vt == VELOXQ_I32);
    if (integer && ch)
        for (int64_t i = 0; i < ctx->n; ++i)
            if (!(std::fabs(ch[i]) < 4.0e15) || ch[i] != std::floor(ch[i])) { integer = false; break; }
    if (ch)
        for (int64_t i = 0; i < ctx->n; ++i)
            if (!std::isfinite(ch[i])) return fail(VELOXQ_EINVAL, "linear term holds a non-finite value");
    ctx->integer = integer;
    switch (vt) {
        case VELOXQ_I8: return ingest_csr_t<int8_t>(ctx, rowptr, col, val, ch, ising, integer);
        case VELOXQ_I32: return ingest_csr_t<int32_t>(ctx, rowptr, col, val, ch, ising, integer);
        case VELOXQ_F32: return ingest_csr_t<float>(ctx, rowptr, col, val, ch, ising, integer);
        case VELOXQ_F64: return ingest_csr_t<double>(ctx, rowptr, col, val, ch, ising, integer);
    }
    return fail(VELOXQ_EINVAL, "unknown value type");
}

// rho(Qoff): by power iteration in one CTA for small sparse instances
// (w_t = Qoff (w_{t-1} / |w_{t-1}|), rho ~ |w_T| after `iters` iterations), by
// kLzSteps steps of Lanczos otherwise.
int power_iteration(veloxq_ctx* ctx, int iters, double* rho) {
    const int64_t n = ctx->n;
    cudaStream_t st = ctx->stream;
    double h = 0.0;
    // slots per row of the one-CTA form: the longest row rounded up to 6, 8,
    // 12 or 16 (0: CSR rows)
    int W = 0;
    for (int c : {6, 8, 12, 16})
        if (ctx->max_row <= c) {
            W = c;
            break;
        }
    if (W && pi_smem(n, ctx->nnz, W) > kPiSmemMax) W = 0;
    if (!ctx->dense && ctx->has_csr && n <= kPiSingleMaxN && pi_smem(n, ctx->nnz, W) <= kPiSmemMax) {
        DevBuf one;
        VQ_TRY(one.ensure(sizeof(double)));
        const size_t sm = pi_smem(n, ctx->nnz, W);
        void (*fn)(int32_t, int32_t, int, const int64_t*, const int32_t*, const float*, double*) =
            W == 6 ? k_pi_single<6> : W == 8 ? k_pi_single<8> : W == 12 ? k_pi_single<12>
                                    : W == 16 ? k_pi_single<16> : k_pi_single<0>;
        VQ_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        fn<<<1, kPiThreads, sm, st>>>((int32_t)n, (int32_t)ctx->nnz, iters, ctx->rowptr.as<int64_t>(),
                                      ctx->col.as<int32_t>(), ctx->wf.as<float>(), one.as<double>());
        VQ_LAUNCH_CHECK("power iteration");
        VQ_CUDA(cudaMemcpyAsync(&h, one.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        VQ_CUDA(cudaStreamSynchronize(st));
        *rho = std::sqrt(h);
        return VELOXQ_OK;
    }
    const int64_t grid_cap = (int64_t)device_sms(ctx->device) * (2048 / kPiBlock);
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(ctx->dense ? div_up(n, kPiBlock / 32) : div_up(n, kPiBlock), grid_cap));
    // the vector update touches n elements: one thread each, no more blocks
    // (a dense matrix pass has a warp per row, 32 times as many threads,
    // and a block count that large only lengthens the update's reduction)
    const unsigned ugrid = (unsigned)std::min<int64_t>(grid, std::max<int64_t>(1, div_up(n, kPiBlock)));
    const int m = (int)std::min<int64_t>(kLzSteps, n);
    DevBuf buf;
    const size_t vbytes = (sizeof(float) * (size_t)(3 * n) + 15) & ~size_t(15);
    VQ_TRY(buf.ensure(vbytes + sizeof(double) * ((size_t)grid + 2 * kLzSteps + 4) + 16));
    float* wv[3] = {buf.as<float>(), buf.as<float>() + n, buf.as<float>() + 2 * n};
    LzScal sc;
    sc.part = reinterpret_cast<double*>(buf.as<uint8_t>() + vbytes);
    sc.alpha = sc.part + grid;
    sc.nrm2 = sc.alpha + kLzSteps;
    sc.count = reinterpret_cast<unsigned*>(sc.nrm2 + kLzSteps + 2);
    VQ_CUDA(cudaMemsetAsync(sc.count, 0, sizeof(unsigned), st));
    k_lz_start<<<grid, kPiBlock, 0, st>>>(n, wv[0], sc);
    for (int j = 0; j < m; ++j) {
        float* wj = wv[j % 3];
        float* u = wv[(j + 1) % 3];
        if (ctx->dense)
            k_lz_gemv<<<grid, kPiBlock, 0, st>>>(n, ctx->qoff32.as<float>(), wj, u, sc, j);
        else
            k_lz_spmv<<<grid, kPiBlock, 0, st>>>(n, ctx->rowptr.as<int64_t>(), ctx->col.as<int32_t>(),
                                                 ctx->wf.as<float>(), wj, u, sc, j);
        if (j + 1 < m) k_lz_update<<<ugrid, kPiBlock, 0, st>>>(n, u, wj, wv[(j + 2) % 3], sc, j);
    }
    VQ_LAUNCH_CHECK("Lanczos");
    std::vector<double> al((size_t)m), n2((size_t)m);
    VQ_CUDA(cudaMemcpyAsync(al.data(), sc.alpha, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    VQ_CUDA(cudaMemcpyAsync(n2.data(), sc.nrm2, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    VQ_CUDA(cudaStreamSynchronize(st));
    std::vector<double> be((size_t)std::max(0, m - 1));
    for (int j = 0; j + 1 < m; ++j) be[j] = std::sqrt(std::max(0.0, n2[j + 1]));
    double lo = 0.0, hi = 0.0;
    tridiag_extremes(al, be, &lo, &hi);
    *rho = std::max(std::fabs(lo), std::fabs(hi));
    return VELOXQ_OK;
}

}  // namespace vq
