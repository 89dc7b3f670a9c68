/*
 * oracle.c -- plain, slow, single-threaded FP64 reference of the VeloxQ hot
 * path (arXiv:2501.19221). TEST INFRASTRUCTURE ONLY: the tests, the smoke
 * check and the CPU-baseline leg of the benchmark call it; the library never
 * does. It shares no code, header or table with the CUDA library.
 *
 * Conventions (each one is a reading of the paper, listed with its reason in
 * the design notes of the repository):
 *
 *  - QUBO energy, Sec. 2 eq. (qubo_model), read as the sum over every stored
 *    entry:   E(x) = sum_{i,j} Q_ij x_i x_j + sum_i c_i x_i.
 *  - Ising energy, Sec. 2 eq. (ising_model):
 *             H(s) = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i   (J read from its
 *    strict upper triangle).
 *  - Dynamics: the simulated-bifurcation equations of App. B (eqs. sbm2, sbm)
 *    in their ballistic form: the quartic term is dropped and inelastic walls
 *    at |s| = 1 are added. With the symmetric part Qs = (Q + Q^T)/2, its
 *    off-diagonal part Qoff and b = Qs 1 + c, one step k of K is
 *        F     = Qoff s
 *        phi   = -(F + b)/2
 *        y    <- y + dt (-(a0 - a_k) s + c0 phi)
 *        s    <- s + dt a0 y
 *        |s| > 1  =>  s <- sign(s), y <- 0
 *    and the readout (App. B: s_i = sign(q_i)) is x = [s > 0].
 *  - a_k is the piecewise-linear interpolation of n_knots values spread
 *    evenly over steps 0 .. K-1 (App. B: a(t) increases linearly through the
 *    bifurcation at a(t) ~ a0); the default knots {0, a0} give a_k = a0 k/(K-1).
 *  - Initial state: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
 *    counter (i_lo, i_hi, r, 0) and key (seed_lo, seed_hi); word 0 draws s,
 *    word 1 draws y; u = (w >> 8) 2^-24 and v = sigma0 (2u - 1) in float32.
 *
 *  - Two further integrators on the same field (method codes 1 and 2):
 *    adiabatic SB exactly as App. B prints it (the quartic potential term,
 *    no walls):
 *        y    <- y + dt (-(s^2 + a0 - a_k) s + c0 phi),  s <- s + dt a0 y
 *    and Parallel Annealing (App. B, "PA"): analog spins x in [-1, 1], the
 *    target gradient taken at the binarised spins sigma = sign(x) (read as
 *    +1 for x > 0 and -1 otherwise, the same rule as the readout), the
 *    initial Hamiltonian sum x^2/2 weighted by lambda_k, momentum and
 *    clipping:
 *        F     = Qoff sigma,  g = lambda_k x + c0 (F + b)/2  (= lambda_k x - c0 phi)
 *        m    <- alpha m - dt g,  x <- clip(x + m, -1, 1)
 *    with lambda_k = (a0 - a_k)/a0 falling from 1 to 0 along the same
 *    schedule. (x, m) use the storage of (s, y); the readout is x = [x > 0].
 *
 * All state arrays are replica-major: element (r, i) lives at r*n + i.
 * Couplings are passed as a coordinate list (er, ec, ev): every stored entry
 * of Q, diagonal included, exactly as given.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the published definition (SC'11, Sec. 3 and Table 2) */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Initial state s0, y0 ~ U(-sigma0, sigma0), exact float32 values. */
void oracle_init_state(int64_t n, int32_t R, uint64_t seed, float sigma0, float* S0, float* Y0)
{
    const uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (int32_t r = 0; r < R; ++r) {
        for (int64_t i = 0; i < n; ++i) {
            uint32_t ctr[4] = { (uint32_t)i, (uint32_t)((uint64_t)i >> 32), (uint32_t)r, 0u };
            uint32_t w[4];
            oracle_philox4x32_10(ctr, key, w);
            /* u = m 2^-24 with m < 2^24; 2u - 1 is exact in float32 */
            float us = (float)(w[0] >> 8) * 5.9604644775390625e-8f;
            float uy = (float)(w[1] >> 8) * 5.9604644775390625e-8f;
            float vs = 2.0f * us - 1.0f;
            float vy = 2.0f * uy - 1.0f;
            volatile float ps = sigma0 * vs;   /* one float32 rounding each */
            volatile float py = sigma0 * vy;
            S0[(int64_t)r * n + i] = ps;
            Y0[(int64_t)r * n + i] = py;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Energies, Sec. 2 eq. (qubo_model) summed over every stored entry           */
/* ------------------------------------------------------------------------ */
int64_t oracle_energy_i64(int64_t n, int64_t nnz, const int64_t* er, const int64_t* ec,
                          const int64_t* ev, const int64_t* c, const uint8_t* x)
{
    int64_t E = 0;
    for (int64_t e = 0; e < nnz; ++e)
        if (x[er[e]] && x[ec[e]]) E += ev[e];
    if (c)
        for (int64_t i = 0; i < n; ++i)
            if (x[i]) E += c[i];
    return E;
}

double oracle_energy_f64(int64_t n, int64_t nnz, const int64_t* er, const int64_t* ec,
                         const double* ev, const double* c, const uint8_t* x)
{
    double E = 0.0;
    for (int64_t e = 0; e < nnz; ++e)
        if (x[er[e]] && x[ec[e]]) E += ev[e];
    if (c)
        for (int64_t i = 0; i < n; ++i)
            if (x[i]) E += c[i];
    return E;
}

/* Batched wrappers: X is [B][n]. */
void oracle_energy_batch_i64(int64_t n, int64_t nnz, const int64_t* er, const int64_t* ec,
                             const int64_t* ev, const int64_t* c, int64_t B, const uint8_t* X, int64_t* E)
{
    for (int64_t b = 0; b < B; ++b) E[b] = oracle_energy_i64(n, nnz, er, ec, ev, c, X + b * n);
}

void oracle_energy_batch_f64(int64_t n, int64_t nnz, const int64_t* er, const int64_t* ec,
                             const double* ev, const double* c, int64_t B, const uint8_t* X, double* E)
{
    for (int64_t b = 0; b < B; ++b) E[b] = oracle_energy_f64(n, nnz, er, ec, ev, c, X + b * n);
}

/* Exhaustive minimum over all 2^n binary vectors (n <= 30). x is the bit
 * pattern of the assignment (bit i = x_i). Returns the first minimiser in
 * increasing bit-pattern order and how many assignments attain the minimum. */
int64_t oracle_bruteforce_i64(int64_t n, int64_t nnz, const int64_t* er, const int64_t* ec,
                              const int64_t* ev, const int64_t* c, uint64_t* argmin, int64_t* count_min)
{
    uint8_t* x = (uint8_t*)calloc((size_t)n, 1);
    int64_t best = INT64_MAX, cnt = 0;
    uint64_t arg = 0;
    const uint64_t total = (uint64_t)1 << n;
    for (uint64_t m = 0; m < total; ++m) {
        for (int64_t i = 0; i < n; ++i) x[i] = (uint8_t)((m >> i) & 1u);
        int64_t E = oracle_energy_i64(n, nnz, er, ec, ev, c, x);
        if (E < best) { best = E; arg = m; cnt = 1; }
        else if (E == best) ++cnt;
    }
    free(x);
    if (argmin) *argmin = arg;
    if (count_min) *count_min = cnt;
    return best;
}

double oracle_bruteforce_f64(int64_t n, int64_t nnz, const int64_t* er, const int64_t* ec,
                             const double* ev, const double* c, uint64_t* argmin)
{
    uint8_t* x = (uint8_t*)calloc((size_t)n, 1);
    double best = INFINITY;
    uint64_t arg = 0;
    const uint64_t total = (uint64_t)1 << n;
    for (uint64_t m = 0; m < total; ++m) {
        for (int64_t i = 0; i < n; ++i) x[i] = (uint8_t)((m >> i) & 1u);
        double E = oracle_energy_f64(n, nnz, er, ec, ev, c, x);
        if (E < best) { best = E; arg = m; }
    }
    free(x);
    if (argmin) *argmin = arg;
    return best;
}

/* Ising energy, Sec. 2 eq. (ising_model): J dense n x n, strict upper triangle. */
double oracle_ising_energy(int64_t n, const double* J, const double* h, const int8_t* s)
{
    double H = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            H += J[i * n + j] * (double)s[i] * (double)s[j];
    for (int64_t i = 0; i < n; ++i) H += h[i] * (double)s[i];
    return H;
}

/* Third-order Ising cost function (Sec. "HUBO", eqs. nn and mw3s):
 *   H(s) = sum_i h_i s_i + sum_q J_q s_pi s_pj + sum_q K_q s_ti s_tj s_tk
 * for one spin vector s in {-1, +1}^n (h may be NULL). */
double oracle_hubo3_energy(int64_t n, const double* h, int64_t n2, const int64_t* pi, const int64_t* pj,
                           const double* J2, int64_t n3, const int64_t* ti, const int64_t* tj, const int64_t* tk,
                           const double* K3, const int8_t* s)
{
    double H = 0.0;
    if (h)
        for (int64_t i = 0; i < n; ++i) H += h[i] * (double)s[i];
    for (int64_t q = 0; q < n2; ++q) H += J2[q] * (double)s[pi[q]] * (double)s[pj[q]];
    for (int64_t q = 0; q < n3; ++q) H += K3[q] * (double)s[ti[q]] * (double)s[tj[q]] * (double)s[tk[q]];
    return H;
}

/* Reduction to second order (Sec. "HUBO", eq. reduction): each cubic term
 * K s_i s_j s_k gets an auxiliary spin a = s_{n+q} and is replaced by
 *   |K| [3 + sgn(K)(s_i + s_j + s_k + 2a) + 2a(s_i + s_j + s_k)
 *        + s_i s_j + s_j s_k + s_i s_k].
 * Output: the pair list (input pairs first, then six per cubic term, not
 * merged; capacity n2 + 6 n3), the fields lin (n + n3; h may be NULL) and
 * the constant. */
void oracle_hubo3_reduce(int64_t n, const double* h, int64_t n2, const int64_t* pi, const int64_t* pj,
                         const double* J2, int64_t n3, const int64_t* ti, const int64_t* tj, const int64_t* tk,
                         const double* K3, int64_t* qi, int64_t* qj, double* qv, double* lin, double* offset)
{
    int64_t m = 0;
    for (int64_t q = 0; q < n2; ++q) { qi[m] = pi[q]; qj[m] = pj[q]; qv[m] = J2[q]; ++m; }
    for (int64_t i = 0; i < n + n3; ++i) lin[i] = (h && i < n) ? h[i] : 0.0;
    double off = 0.0;
    for (int64_t q = 0; q < n3; ++q) {
        int64_t t[3] = {ti[q], tj[q], tk[q]};
        int64_t a = n + q;
        double K = K3[q], absK = fabs(K), sg = K > 0.0 ? 1.0 : (K < 0.0 ? -1.0 : 0.0);
        off += 3.0 * absK;
        for (int u = 0; u < 3; ++u) {
            lin[t[u]] += sg * absK;                             /* sgn(K)|K| s_u */
            qi[m] = a; qj[m] = t[u]; qv[m] = 2.0 * absK; ++m;   /* 2|K| a s_u */
        }
        lin[a] += 2.0 * sg * absK;                              /* 2 sgn(K)|K| a */
        qi[m] = t[0]; qj[m] = t[1]; qv[m] = absK; ++m;
        qi[m] = t[1]; qj[m] = t[2]; qv[m] = absK; ++m;
        qi[m] = t[0]; qj[m] = t[2]; qv[m] = absK; ++m;
    }
    *offset = off;
}

/* ------------------------------------------------------------------------ */
/* App. A conversions (dense)                                                */
/* ------------------------------------------------------------------------ */
/* Ising -> QUBO (App. A, eq. qij_SK): Q_ij = J_ij (i != j, symmetric, from
 * the strict upper triangle), Q_ii = h_i - sum_l J_il. H(s) = 2 Q(x) + C with
 * C = sum_{i<j} J_ij - sum_i h_i (the sign derived from x = (1 + s)/2; the
 * paper prints the opposite sign). */
void oracle_ising_to_qubo(int64_t n, const double* J, const double* h, double* Q, double* C)
{
    double sumJ = 0.0, sumh = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) Q[i * n + j] = 0.0;
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            Q[i * n + j] = J[i * n + j];
            Q[j * n + i] = J[i * n + j];
            sumJ += J[i * n + j];
        }
    for (int64_t i = 0; i < n; ++i) {
        double row = 0.0;
        for (int64_t l = 0; l < n; ++l)
            if (l != i) row += Q[i * n + l];
        Q[i * n + i] = h[i] - row;
        sumh += h[i];
    }
    *C = sumJ - sumh;
}

/* QUBO -> Ising (App. A, eq. Jh_QUBO): h_i = sum_j Q_ij, J_ij = Q_ij (i != j),
 * for symmetric Q; Q(x) = H(s)/2 + C/2 with C = sum_{i<j} Q_ij + sum_i Q_ii
 * (the sign derived from x = (1 + s)/2; the paper prints -C/2). */
void oracle_qubo_to_ising(int64_t n, const double* Q, double* J, double* h, double* C)
{
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double hi = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            hi += Q[i * n + j];
            J[i * n + j] = (i == j) ? 0.0 : Q[i * n + j];
            if (j > i) acc += Q[i * n + j];
        }
        h[i] = hi;
        acc += Q[i * n + i];
    }
    *C = acc;
}

/* ------------------------------------------------------------------------ */
/* Normalisation and local field                                             */
/* ------------------------------------------------------------------------ */
/* b = Qs 1 + c and K0 = 1/4 1^T Qoff 1 + 1/2 tr Q + 1/2 sum c, so that
 * E(x) = 1/4 s^T Qoff s + 1/2 b^T s + K0 for s = 2x - 1. */
void oracle_bias(int64_t n, int64_t nnz, const int64_t* er, const int64_t* ec, const double* ev,
                 const double* c, double* b, double* K0)
{
    double k0 = 0.0;
    for (int64_t i = 0; i < n; ++i) b[i] = c ? c[i] : 0.0;
    for (int64_t e = 0; e < nnz; ++e) {
        int64_t i = er[e], j = ec[e];
        if (i == j) {
            b[i] += ev[e];
            k0 += 0.5 * ev[e];
        } else {
            b[i] += 0.5 * ev[e];
            b[j] += 0.5 * ev[e];
            k0 += 0.25 * ev[e];
        }
    }
    if (c)
        for (int64_t i = 0; i < n; ++i) k0 += 0.5 * c[i];
    *K0 = k0;
}

/* F = Qoff S with Qoff = off-diagonal part of (Q + Q^T)/2; S, F are [R][n]. */
void oracle_field(int64_t n, int64_t nnz, const int64_t* er, const int64_t* ec, const double* ev,
                  int32_t R, const double* S, double* F)
{
    for (int32_t r = 0; r < R; ++r) {
        const double* s = S + (int64_t)r * n;
        double* f = F + (int64_t)r * n;
        for (int64_t i = 0; i < n; ++i) f[i] = 0.0;
        for (int64_t e = 0; e < nnz; ++e) {
            int64_t i = er[e], j = ec[e];
            if (i == j) continue;
            f[i] += 0.5 * ev[e] * s[j];
            f[j] += 0.5 * ev[e] * s[i];
        }
    }
}

/* a_k for k = 0 .. K-1 from n_knots evenly spread knots. */
void oracle_schedule(int32_t K, int32_t n_knots, const double* knots, double* a)
{
    for (int32_t k = 0; k < K; ++k) {
        if (K == 1 || n_knots == 1) { a[k] = knots[0]; continue; }
        double t = (double)k * (double)(n_knots - 1) / (double)(K - 1);
        int32_t j = (int32_t)floor(t);
        if (j > n_knots - 2) j = n_knots - 2;
        double w = t - (double)j;
        a[k] = knots[j] * (1.0 - w) + knots[j + 1] * w;
    }
}

/* Interpolation weight of knot j in a_k (same rule as oracle_schedule). */
static double knot_weight(int32_t K, int32_t n_knots, int32_t k, int32_t j)
{
    if (K == 1 || n_knots == 1) return j == 0 ? 1.0 : 0.0;
    double t = (double)k * (double)(n_knots - 1) / (double)(K - 1);
    int32_t lo = (int32_t)floor(t);
    if (lo > n_knots - 2) lo = n_knots - 2;
    double w = t - (double)lo;
    if (j == lo) return 1.0 - w;
    if (j == lo + 1) return w;
    return 0.0;
}

/* One ballistic-SB update (App. B eqs. sbm2/sbm without the quartic term,
 * plus walls), given the field F of the current state. In place on S, Y. */
void oracle_bsb_update(int64_t n, int32_t R, const double* F, const double* b, double a_k,
                       double dt, double a0, double c0, double* S, double* Y)
{
    for (int32_t r = 0; r < R; ++r)
        for (int64_t i = 0; i < n; ++i) {
            int64_t p = (int64_t)r * n + i;
            double phi = -0.5 * (F[p] + b[i]);
            double y = Y[p] + dt * (-(a0 - a_k) * S[p] + c0 * phi);
            double s = S[p] + dt * a0 * y;
            if (fabs(s) > 1.0) { s = s > 0.0 ? 1.0 : -1.0; y = 0.0; }
            S[p] = s;
            Y[p] = y;
        }
}

/* One adiabatic-SB update as App. B prints it (eq. sbm with the quartic
 * potential, no walls), given the field F of the current state. */
void oracle_asb_update(int64_t n, int32_t R, const double* F, const double* b, double a_k,
                       double dt, double a0, double c0, double* S, double* Y)
{
    for (int32_t r = 0; r < R; ++r)
        for (int64_t i = 0; i < n; ++i) {
            int64_t p = (int64_t)r * n + i;
            double s = S[p];
            double phi = -0.5 * (F[p] + b[i]);
            double y = Y[p] + dt * (-(s * s + a0 - a_k) * s + c0 * phi);
            S[p] = s + dt * a0 * y;
            Y[p] = y;
        }
}

/* One Parallel-Annealing update (App. B: gradient step with momentum and
 * clipping on the analog spins), given the field F of the binarised spins
 * and lambda_k. X holds the analog spins, M the momenta. */
void oracle_pa_update(int64_t n, int32_t R, const double* F, const double* b, double lam,
                      double dt, double alpha, double c0, double* X, double* M)
{
    for (int32_t r = 0; r < R; ++r)
        for (int64_t i = 0; i < n; ++i) {
            int64_t p = (int64_t)r * n + i;
            double g = lam * X[p] + c0 * 0.5 * (F[p] + b[i]);
            double m = alpha * M[p] - dt * g;
            double x = X[p] + m;
            if (x > 1.0) x = 1.0;
            if (x < -1.0) x = -1.0;
            X[p] = x;
            M[p] = m;
        }
}

/* The field operand of a method: the state itself (SB forms) or its
 * binarised spins, +1 where x > 0 and -1 elsewhere (PA). */
void oracle_field_operand(int32_t method, int64_t nR, const double* S, double* out)
{
    for (int64_t p = 0; p < nR; ++p) out[p] = method == 2 ? (S[p] > 0.0 ? 1.0 : -1.0) : S[p];
}

/* One update of the given method (0 ballistic SB, 1 adiabatic SB, 2 PA). */
void oracle_update(int32_t method, int64_t n, int32_t R, const double* F, const double* b, double a_k,
                   double dt, double a0, double c0, double alpha, double* S, double* Y)
{
    if (method == 1) oracle_asb_update(n, R, F, b, a_k, dt, a0, c0, S, Y);
    else if (method == 2) oracle_pa_update(n, R, F, b, (a0 - a_k) / a0, dt, alpha, c0, S, Y);
    else oracle_bsb_update(n, R, F, b, a_k, dt, a0, c0, S, Y);
}

/* ------------------------------------------------------------------------ */
/* Full run with readout, exact energy and best-so-far                        */
/* ------------------------------------------------------------------------ */
/* Runs K steps from (S0, Y0). After step k (count k+1) a readout happens when
 * (k+1) % readout_every == 0 (readout_every > 0) and always after the last
 * step. Each replica keeps the first strictly lowest energy it reads out.
 * ev_i64/c_i64 (may be NULL) switch the energy to exact int64.
 * Snapshots (if n_snap > 0): F_snap[k] is the field used in step k, S_snap[k]
 * and Y_snap[k] the state after step k, each [R][n], for k < n_snap. */
/* The run of any method (0 ballistic SB, 1 adiabatic SB, 2 PA; alpha is
 * the PA momentum). For PA the snapshots F_snap hold the field of the
 * binarised spins. */
int oracle_run(int32_t method, double alpha,
               int64_t n, int64_t nnz, const int64_t* er, const int64_t* ec, const double* ev,
               const double* c, const int64_t* ev_i64, const int64_t* c_i64,
               int32_t R, int32_t K, double dt, double a0, double c0,
               int32_t n_knots, const double* knots, int32_t readout_every,
               const float* S0, const float* Y0,
               int32_t n_snap, double* F_snap, double* S_snap, double* Y_snap,
               double* S_fin, double* Y_fin,
               double* best_E, int64_t* best_E_i64, uint8_t* best_x, int32_t* best_step)
{
    const int64_t nR = n * (int64_t)R;
    double* S = (double*)malloc(sizeof(double) * (size_t)nR);
    double* Y = (double*)malloc(sizeof(double) * (size_t)nR);
    double* F = (double*)malloc(sizeof(double) * (size_t)nR);
    double* O = (double*)malloc(sizeof(double) * (size_t)nR);
    double* b = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* a = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
    uint8_t* x = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
    if (!S || !Y || !F || !O || !b || !a || !x) return -2;
    double K0;
    oracle_bias(n, nnz, er, ec, ev, c, b, &K0);
    oracle_schedule(K, n_knots, knots, a);
    for (int64_t p = 0; p < nR; ++p) { S[p] = (double)S0[p]; Y[p] = (double)Y0[p]; }
    for (int32_t r = 0; r < R; ++r) {
        best_E[r] = INFINITY;
        if (best_E_i64) best_E_i64[r] = INT64_MAX;
        if (best_step) best_step[r] = -1;
    }
    for (int32_t k = 0; k < K; ++k) {
        oracle_field_operand(method, nR, S, O);
        oracle_field(n, nnz, er, ec, ev, R, O, F);
        if (k < n_snap && F_snap) memcpy(F_snap + (int64_t)k * nR, F, sizeof(double) * (size_t)nR);
        oracle_update(method, n, R, F, b, a[k], dt, a0, c0, alpha, S, Y);
        if (k < n_snap && S_snap) memcpy(S_snap + (int64_t)k * nR, S, sizeof(double) * (size_t)nR);
        if (k < n_snap && Y_snap) memcpy(Y_snap + (int64_t)k * nR, Y, sizeof(double) * (size_t)nR);
        int readout = (k == K - 1) || (readout_every > 0 && ((k + 1) % readout_every) == 0);
        if (!readout) continue;
        for (int32_t r = 0; r < R; ++r) {
            for (int64_t i = 0; i < n; ++i) x[i] = S[(int64_t)r * n + i] > 0.0 ? 1 : 0;
            int improved;
            if (ev_i64) {
                int64_t E = oracle_energy_i64(n, nnz, er, ec, ev_i64, c_i64, x);
                improved = E < best_E_i64[r];
                if (improved) { best_E_i64[r] = E; best_E[r] = (double)E; }
            } else {
                double E = oracle_energy_f64(n, nnz, er, ec, ev, c, x);
                improved = E < best_E[r];
                if (improved) best_E[r] = E;
            }
            if (improved) {
                if (best_x) memcpy(best_x + (int64_t)r * n, x, (size_t)n);
                if (best_step) best_step[r] = k + 1;
            }
        }
    }
    if (S_fin) memcpy(S_fin, S, sizeof(double) * (size_t)nR);
    if (Y_fin) memcpy(Y_fin, Y, sizeof(double) * (size_t)nR);
    free(S); free(Y); free(F); free(O); free(b); free(a); free(x);
    return 0;
}

/* The ballistic-SB run (method 0). */
int oracle_bsb_run(int64_t n, int64_t nnz, const int64_t* er, const int64_t* ec, const double* ev,
                   const double* c, const int64_t* ev_i64, const int64_t* c_i64,
                   int32_t R, int32_t K, double dt, double a0, double c0,
                   int32_t n_knots, const double* knots, int32_t readout_every,
                   const float* S0, const float* Y0,
                   int32_t n_snap, double* F_snap, double* S_snap, double* Y_snap,
                   double* S_fin, double* Y_fin,
                   double* best_E, int64_t* best_E_i64, uint8_t* best_x, int32_t* best_step)
{
    return oracle_run(0, 0.0, n, nnz, er, ec, ev, c, ev_i64, c_i64, R, K, dt, a0, c0, n_knots, knots,
                      readout_every, S0, Y0, n_snap, F_snap, S_snap, Y_snap, S_fin, Y_fin, best_E, best_E_i64,
                      best_x, best_step);
}

/* Relaxed energy per replica: 1/4 s^T Qoff s + 1/2 b^T s + K0 (identity of
 * the QUBO energy under x = (1 + s)/2, evaluated at a continuous s). */
void oracle_relaxed_energy(int64_t n, int64_t nnz, const int64_t* er, const int64_t* ec, const double* ev,
                           const double* c, int32_t R, const double* S, double* E)
{
    double* b = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* F = (double*)malloc(sizeof(double) * (size_t)(n * (int64_t)R > 0 ? n * (int64_t)R : 1));
    double K0;
    oracle_bias(n, nnz, er, ec, ev, c, b, &K0);
    oracle_field(n, nnz, er, ec, ev, R, S, F);
    for (int32_t r = 0; r < R; ++r) {
        double acc = K0;
        for (int64_t i = 0; i < n; ++i) {
            int64_t p = (int64_t)r * n + i;
            acc += 0.25 * S[p] * F[p] + 0.5 * b[i] * S[p];
        }
        E[r] = acc;
    }
    free(b); free(F);
}

/* ------------------------------------------------------------------------ */
/* Reverse-mode gradient of L = mean_r E_relax(s_K) through K unrolled steps  */
/* ------------------------------------------------------------------------ */
/* Stores the whole trajectory (small cases only). Returns L and dL/d(dt),
 * dL/d(c0) and dL/d(knot_j). Where the wall is active the step's outputs are
 * constants (sign and 0), so no gradient passes through them. */
int oracle_bsb_grad(int64_t n, int64_t nnz, const int64_t* er, const int64_t* ec, const double* ev,
                    const double* c, int32_t R, int32_t K, double dt, double a0, double c0,
                    int32_t n_knots, const double* knots, const float* S0, const float* Y0,
                    double* loss, double* d_dt, double* d_c0, double* d_knots)
{
    const int64_t nR = n * (int64_t)R;
    double* Ss = (double*)malloc(sizeof(double) * (size_t)nR * (size_t)(K + 1));
    double* Ys = (double*)malloc(sizeof(double) * (size_t)nR * (size_t)(K + 1));
    double* F = (double*)malloc(sizeof(double) * (size_t)nR);
    double* G = (double*)malloc(sizeof(double) * (size_t)nR);   /* Qoff applied to g_phi */
    double* gphi = (double*)malloc(sizeof(double) * (size_t)nR);
    double* ls = (double*)malloc(sizeof(double) * (size_t)nR);
    double* ly = (double*)malloc(sizeof(double) * (size_t)nR);
    double* b = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* a = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
    double* da = (double*)calloc((size_t)(K > 0 ? K : 1), sizeof(double));
    if (!Ss || !Ys || !F || !G || !gphi || !ls || !ly || !b || !a || !da) return -2;
    double K0;
    oracle_bias(n, nnz, er, ec, ev, c, b, &K0);
    oracle_schedule(K, n_knots, knots, a);
    for (int64_t p = 0; p < nR; ++p) { Ss[p] = (double)S0[p]; Ys[p] = (double)Y0[p]; }
    /* forward, keeping every state */
    for (int32_t k = 0; k < K; ++k) {
        double* S = Ss + (int64_t)(k + 1) * nR;
        double* Y = Ys + (int64_t)(k + 1) * nR;
        memcpy(S, Ss + (int64_t)k * nR, sizeof(double) * (size_t)nR);
        memcpy(Y, Ys + (int64_t)k * nR, sizeof(double) * (size_t)nR);
        oracle_field(n, nnz, er, ec, ev, R, Ss + (int64_t)k * nR, F);
        oracle_bsb_update(n, R, F, b, a[k], dt, a0, c0, S, Y);
    }
    /* loss and its gradient w.r.t. s_K: (Qoff s + b) / (2R) */
    const double* SK = Ss + (int64_t)K * nR;
    oracle_field(n, nnz, er, ec, ev, R, SK, F);
    double L = 0.0;
    for (int32_t r = 0; r < R; ++r) {
        double acc = K0;
        for (int64_t i = 0; i < n; ++i) {
            int64_t p = (int64_t)r * n + i;
            acc += 0.25 * SK[p] * F[p] + 0.5 * b[i] * SK[p];
            ls[p] = (0.5 * F[p] + 0.5 * b[i]) / (double)R;
            ly[p] = 0.0;
        }
        L += acc;
    }
    L /= (double)R;
    double gdt = 0.0, gc0 = 0.0;
    /* reverse sweep */
    for (int32_t k = K - 1; k >= 0; --k) {
        const double* S = Ss + (int64_t)k * nR;
        const double* Y = Ys + (int64_t)k * nR;
        oracle_field(n, nnz, er, ec, ev, R, S, F);
        for (int32_t r = 0; r < R; ++r)
            for (int64_t i = 0; i < n; ++i) {
                int64_t p = (int64_t)r * n + i;
                double phi = -0.5 * (F[p] + b[i]);
                double drive = -(a0 - a[k]) * S[p] + c0 * phi;
                double yh = Y[p] + dt * drive;
                double sh = S[p] + dt * a0 * yh;
                int wall = fabs(sh) > 1.0;
                double g_sh = wall ? 0.0 : ls[p];
                double g_yh = wall ? 0.0 : ly[p];
                /* sh = s + dt a0 yh */
                double g_s = g_sh;
                g_yh += dt * a0 * g_sh;
                gdt += a0 * yh * g_sh;
                /* yh = y + dt (-(a0 - a_k) s + c0 phi) */
                double g_y = g_yh;
                g_s += -dt * (a0 - a[k]) * g_yh;
                gphi[p] = dt * c0 * g_yh;
                gdt += drive * g_yh;
                da[k] += dt * S[p] * g_yh;
                gc0 += dt * phi * g_yh;
                ls[p] = g_s;          /* the -Qoff g_phi / 2 part is added below */
                ly[p] = g_y;
            }
        /* phi = -(Qoff s + b)/2  =>  g_s += -Qoff g_phi / 2 (Qoff symmetric) */
        oracle_field(n, nnz, er, ec, ev, R, gphi, G);
        for (int64_t p = 0; p < nR; ++p) ls[p] += -0.5 * G[p];
    }
    *loss = L;
    *d_dt = gdt;
    *d_c0 = gc0;
    for (int32_t j = 0; j < n_knots; ++j) {
        double acc = 0.0;
        for (int32_t k = 0; k < K; ++k) acc += knot_weight(K, n_knots, k, j) * da[k];
        d_knots[j] = acc;
    }
    free(Ss); free(Ys); free(F); free(G); free(gphi); free(ls); free(ly); free(b); free(a); free(da);
    return 0;
}

/* Loss only (for finite differences): L = mean_r E_relax(s_K). */
int oracle_bsb_loss(int64_t n, int64_t nnz, const int64_t* er, const int64_t* ec, const double* ev,
                    const double* c, int32_t R, int32_t K, double dt, double a0, double c0,
                    int32_t n_knots, const double* knots, const float* S0, const float* Y0, double* loss)
{
    const int64_t nR = n * (int64_t)R;
    double* S = (double*)malloc(sizeof(double) * (size_t)nR);
    double* Y = (double*)malloc(sizeof(double) * (size_t)nR);
    double* F = (double*)malloc(sizeof(double) * (size_t)nR);
    double* b = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* a = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
    double* E = (double*)malloc(sizeof(double) * (size_t)(R > 0 ? R : 1));
    if (!S || !Y || !F || !b || !a || !E) return -2;
    double K0;
    oracle_bias(n, nnz, er, ec, ev, c, b, &K0);
    oracle_schedule(K, n_knots, knots, a);
    for (int64_t p = 0; p < nR; ++p) { S[p] = (double)S0[p]; Y[p] = (double)Y0[p]; }
    for (int32_t k = 0; k < K; ++k) {
        oracle_field(n, nnz, er, ec, ev, R, S, F);
        oracle_bsb_update(n, R, F, b, a[k], dt, a0, c0, S, Y);
    }
    oracle_relaxed_energy(n, nnz, er, ec, ev, c, R, S, E);
    double L = 0.0;
    for (int32_t r = 0; r < R; ++r) L += E[r];
    *loss = L / (double)R;
    free(S); free(Y); free(F); free(b); free(a); free(E);
    return 0;
}

/* Sparse Ising -> QUBO (App. A, eq. qij_SK) from the coupled pairs (i < j):
 * Q_ij = Q_ji = J_ij and Q_ii = h_i - sum_l J_il, written as a coordinate list
 * of 2*npairs + n entries (pairs first, then the diagonal); C receives
 * sum_{i<j} J_ij - sum_i h_i so that H(s) = 2 Q(x) + C. */
void oracle_ising_pairs_to_qubo(int64_t n, int64_t npairs, const int64_t* pi, const int64_t* pj, const double* pv,
                                const double* h, int64_t* er, int64_t* ec, double* ev, double* C)
{
    double sumJ = 0.0, sumh = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        er[2 * npairs + i] = i;
        ec[2 * npairs + i] = i;
        ev[2 * npairs + i] = h ? h[i] : 0.0;
        if (h) sumh += h[i];
    }
    for (int64_t e = 0; e < npairs; ++e) {
        er[2 * e] = pi[e]; ec[2 * e] = pj[e]; ev[2 * e] = pv[e];
        er[2 * e + 1] = pj[e]; ec[2 * e + 1] = pi[e]; ev[2 * e + 1] = pv[e];
        ev[2 * npairs + pi[e]] -= pv[e];
        ev[2 * npairs + pj[e]] -= pv[e];
        sumJ += pv[e];
    }
    *C = sumJ - sumh;
}
