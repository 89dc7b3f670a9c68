// vq_hubo.cu -- host-side reduction of a third-order Ising cost function
// (HUBO) to second order, by the gadget of Sec. "HUBO" (eq. reduction):
// one auxiliary spin a per cubic term K s_i s_j s_k, replaced by
//     |K| [ 3 + sgn(K)(s_i + s_j + s_k + 2a) + 2a(s_i + s_j + s_k)
//           + s_i s_j + s_j s_k + s_i s_k ],
// whose minimum over a equals K s_i s_j s_k for every (s_i, s_j, s_k).
// The result is an Ising instance in the CSR form veloxq_create_ising_csr
// takes: structurally symmetric, columns sorted, every pair stored at both
// positions with the same (summed) value.
#include <algorithm>
#include <cmath>
#include <vector>

#include "vq_internal.cuh"

using namespace vq;

// The reduction with every spin v (original v < n, auxiliary n + q) stored at
// index index[v] (a permutation of [0, n + n3)), or at v when index is NULL.
static int reduce3(int64_t n, const double* h, int64_t n2, const int64_t* pi, const int64_t* pj, const double* J2,
                   int64_t n3, const int64_t* ti, const int64_t* tj, const int64_t* tk, const double* K3,
                   int64_t* n_out, int64_t* nnz_out, int64_t* rowptr, int32_t* col, double* val, double* lin,
                   double* offset, const int64_t* index) {
    if (n < 1 || n2 < 0 || n3 < 0) return fail(VELOXQ_EINVAL, "n >= 1, n2 >= 0 and n3 >= 0 required");
    if ((n2 > 0 && (!pi || !pj || !J2)) || (n3 > 0 && (!ti || !tj || !tk || !K3)))
        return fail(VELOXQ_EINVAL, "term arrays must not be NULL");
    if (!n_out || !nnz_out || !rowptr || !col || !val || !lin || !offset)
        return fail(VELOXQ_EINVAL, "output arrays must not be NULL");
    const int64_t N = n + n3;
    if (N > INT32_MAX) return fail(VELOXQ_EINVAL, "n + n3 must fit 32-bit column indices");
    struct Pair {
        int32_t a, b;   // a < b (N fits 32 bits)
        double v;
    };
    std::vector<Pair> pairs;
    pairs.reserve((size_t)(n2 + 6 * n3));
    auto at = [&](int64_t v) { return index ? index[v] : v; };
    auto add = [&](int64_t a, int64_t b, double v) {
        a = at(a);
        b = at(b);
        if (a > b) std::swap(a, b);
        pairs.push_back(Pair{(int32_t)a, (int32_t)b, v});
    };
    for (int64_t q = 0; q < n2; ++q) {
        if (pi[q] < 0 || pi[q] >= n || pj[q] < 0 || pj[q] >= n || pi[q] == pj[q])
            return fail(VELOXQ_EINVAL, "pair " + std::to_string(q) + ": indices out of range or equal");
        if (!std::isfinite(J2[q])) return fail(VELOXQ_EINVAL, "pair coupling is not finite");
        add(pi[q], pj[q], J2[q]);
    }
    for (int64_t i = 0; i < N; ++i) lin[at(i)] = (h && i < n) ? h[i] : 0.0;
    for (int64_t i = 0; i < n && h; ++i)
        if (!std::isfinite(h[i])) return fail(VELOXQ_EINVAL, "field h is not finite");
    double off = 0.0;
    for (int64_t q = 0; q < n3; ++q) {
        const int64_t i = ti[q], j = tj[q], k = tk[q];
        if (i < 0 || i >= n || j < 0 || j >= n || k < 0 || k >= n || i == j || j == k || i == k)
            return fail(VELOXQ_EINVAL, "cubic term " + std::to_string(q) + ": indices out of range or repeated");
        const double K = K3[q];
        if (!std::isfinite(K)) return fail(VELOXQ_EINVAL, "cubic coefficient is not finite");
        const double m = std::fabs(K);
        const int64_t a = n + q;   // the auxiliary spin of this term
        off += 3.0 * m;
        lin[at(i)] += K;           // sgn(K)|K|
        lin[at(j)] += K;
        lin[at(k)] += K;
        lin[at(a)] += 2.0 * K;
        add(a, i, 2.0 * m);
        add(a, j, 2.0 * m);
        add(a, k, 2.0 * m);
        add(i, j, m);
        add(j, k, m);
        add(i, k, m);
    }
    // Sort by (a, b), stably: repeated pairs keep the order of the terms that
    // made them, so their values are summed in that order under any
    // numbering. A stable counting sort by a, then a stable insertion sort by
    // b within each row (rows hold a handful of pairs): the order of one
    // stable sort by (a, b), in linear time.
    {
        std::vector<int64_t> start((size_t)N + 1, 0);
        for (const Pair& p : pairs) ++start[(size_t)p.a + 1];
        for (int64_t i = 0; i < N; ++i) start[(size_t)i + 1] += start[(size_t)i];
        std::vector<Pair> byrow(pairs.size());
        {
            std::vector<int64_t> fill(start.begin(), start.end() - 1);
            for (const Pair& p : pairs) byrow[(size_t)fill[(size_t)p.a]++] = p;
        }
        for (int64_t i = 0; i < N; ++i) {
            Pair* r = byrow.data() + start[(size_t)i];
            const int64_t len = start[(size_t)i + 1] - start[(size_t)i];
            for (int64_t x = 1; x < len; ++x) {
                const Pair key = r[x];
                int64_t y = x - 1;
                while (y >= 0 && r[y].b > key.b) {
                    r[y + 1] = r[y];
                    --y;
                }
                r[y + 1] = key;
            }
        }
        pairs.swap(byrow);
    }
    // merge repeated pairs
    size_t m = 0;
    for (size_t q = 0; q < pairs.size(); ++q) {
        if (m > 0 && pairs[m - 1].a == pairs[q].a && pairs[m - 1].b == pairs[q].b) pairs[m - 1].v += pairs[q].v;
        else pairs[m++] = pairs[q];
    }
    pairs.resize(m);
    // symmetric CSR: per row, the lower entries (ascending) then the upper ones
    std::vector<int64_t> cnt((size_t)N + 1, 0);
    for (const Pair& p : pairs) {
        ++cnt[(size_t)p.a + 1];
        ++cnt[(size_t)p.b + 1];
    }
    for (int64_t i = 0; i < N; ++i) cnt[(size_t)i + 1] += cnt[(size_t)i];
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (const Pair& p : pairs) {   // lower part of row b: column a
        col[fill[(size_t)p.b]] = (int32_t)p.a;
        val[fill[(size_t)p.b]++] = p.v;
    }
    for (const Pair& p : pairs) {   // upper part of row a: column b
        col[fill[(size_t)p.a]] = (int32_t)p.b;
        val[fill[(size_t)p.a]++] = p.v;
    }
    for (int64_t i = 0; i <= N; ++i) rowptr[i] = cnt[(size_t)i];
    *n_out = N;
    *nnz_out = cnt[(size_t)N];
    *offset = off;
    return VELOXQ_OK;
}

extern "C" int veloxq_hubo3_reduce(int64_t n, const double* h, int64_t n2, const int64_t* pi, const int64_t* pj,
                                   const double* J2, int64_t n3, const int64_t* ti, const int64_t* tj,
                                   const int64_t* tk, const double* K3, int64_t* n_out, int64_t* nnz_out,
                                   int64_t* rowptr, int32_t* col, double* val, double* lin, double* offset) {
    return reduce3(n, h, n2, pi, pj, J2, n3, ti, tj, tk, K3, n_out, nnz_out, rowptr, col, val, lin, offset, nullptr);
}

// The same reduction numbered for locality: the original spins in order,
// each followed by the auxiliary spins of the cubic terms whose largest index
// it is (in term order). index[v] is where spin v went.
extern "C" int veloxq_hubo3_reduce_local(int64_t n, const double* h, int64_t n2, const int64_t* pi,
                                         const int64_t* pj, const double* J2, int64_t n3, const int64_t* ti,
                                         const int64_t* tj, const int64_t* tk, const double* K3, int64_t* n_out,
                                         int64_t* nnz_out, int64_t* rowptr, int32_t* col, double* val, double* lin,
                                         double* offset, int64_t* index) {
    if (!index) return fail(VELOXQ_EINVAL, "index must not be NULL");
    if (n < 1 || n3 < 0) return fail(VELOXQ_EINVAL, "n >= 1 and n3 >= 0 required");
    if (n3 > 0 && (!ti || !tj || !tk)) return fail(VELOXQ_EINVAL, "term arrays must not be NULL");
    if (n + n3 > INT32_MAX) return fail(VELOXQ_EINVAL, "n + n3 must fit 32-bit column indices");
    std::vector<int64_t> anchor((size_t)n3), cnt((size_t)n + 1, 0);
    for (int64_t q = 0; q < n3; ++q) {
        const int64_t i = ti[q], j = tj[q], k = tk[q];
        if (i < 0 || i >= n || j < 0 || j >= n || k < 0 || k >= n)
            return fail(VELOXQ_EINVAL, "cubic term " + std::to_string(q) + ": indices out of range or repeated");
        anchor[(size_t)q] = std::max(i, std::max(j, k));
        ++cnt[(size_t)anchor[(size_t)q] + 1];
    }
    // spin v sits after v original spins and the auxiliary spins anchored below v
    for (int64_t v = 0; v < n; ++v) cnt[(size_t)v + 1] += cnt[(size_t)v];
    std::vector<int64_t> next((size_t)n);
    for (int64_t v = 0; v < n; ++v) {
        index[v] = v + cnt[(size_t)v];
        next[(size_t)v] = index[v] + 1;
    }
    for (int64_t q = 0; q < n3; ++q) index[n + q] = next[(size_t)anchor[(size_t)q]]++;
    return reduce3(n, h, n2, pi, pj, J2, n3, ti, tj, tk, K3, n_out, nnz_out, rowptr, col, val, lin, offset, index);
}
