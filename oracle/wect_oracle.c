/*
 * wect_oracle.c -- plain, slow, CPU reference for the weighted Euler characteristic
 * transform (WECT) and function (WECF / ECF) of weighted simplicial and cubical complexes.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load this
 * file; only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code, header or table with the CUDA library.
 *
 * What it computes (the plain definition the method reaches, Section 3, proof of
 * Algorithm 1 and Eq. "ecf"):
 *
 *     W[p][q] = sum over simplices s with bin(max_{v in s} f_p(v)) <= q of (-1)^dim(s) w(s)
 *
 * where f_p is the vertex filter (the height h_s(v) = l(v).s of Definition "Vertex Height
 * Functions" for the WECT, Example "ex:wect"), and bin(t) counts the thresholds beta[q],
 * q <= T-2, strictly below t (the index alpha of Eq. "left-adjoint" read as an exact count,
 * which satisfies the Galois property of Eq. "galois").  The loops follow Algorithm 1's
 * order: the maximum of the vertex values per simplex, its bin, the signed scatter-add of
 * the simplex weight into a difference table, and the cumulative sum over thresholds.
 *
 * Readings of points the paper leaves open:
 *  - heights:  h = x[n-1]*s[n-1], then h = fma(x[c], s[c], h) for c = n-2 .. 0 (float64);
 *  - thresholds: step = (hi-lo)/(T-1), beta[q] = lo + q*step (float64, no contraction);
 *  - bin(t) = #{q in [0, T-2] : beta[q] < t}, so values above hi land in the top bin and
 *    the top column is always the weighted Euler characteristic of the whole complex;
 *  - grid coordinates x_a(i) = (2i - (L_a-1)) / (L_a-1) (0 when L_a = 1), axis 0 fastest;
 *  - cubical cells: every (corner, extent mask) box of the grid; weight = max of its
 *    vertex weights, as in the Figure 1 example; weights are int64 fixed point;
 *  - float weights become rint(w * 2^frac_bits);
 *  - the adjoint routes each simplex's gradient to its heaviest vertex, ties to the lowest
 *    vertex index.
 *
 * Build with -ffp-contract=off so that every multiply and add rounds on its own.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define WO_OK 0
#define WO_ERR 1

/* ---------------------------------------------------------------- primitives */

/* Definition "Vertex Height Functions": h_s(v) = l(v) . s, fixed fma order. */
double wo_height(int n, const double *x, const double *s)
{
    double h = x[n - 1] * s[n - 1];
    for (int c = n - 2; c >= 0; --c) h = fma(x[c], s[c], h);
    return h;
}

/* The discretisation beta(q) = q * 2M/(T-1) - M of Section 3, written for a range [lo, hi]. */
void wo_beta(int T, double lo, double hi, double *beta)
{
    double step = (hi - lo) / (double)(T - 1);
    for (int q = 0; q < T; ++q) beta[q] = lo + (double)q * step;
}

/* alpha of Eq. "left-adjoint" as an exact count: #{q <= T-2 : beta[q] < t}. */
int wo_bin(double t, const double *beta, int T)
{
    int b = 0;
    for (int q = 0; q <= T - 2; ++q)
        if (beta[q] < t) ++b;
    return b;
}

/* Coordinate of grid index i on an axis of length L, scaled to [-1, 1]. */
double wo_grid_coord(int64_t i, int64_t L)
{
    if (L <= 1) return 0.0;
    return (double)(2 * i - (L - 1)) / (double)(L - 1);
}

/* rint(w * 2^frac_bits) for a float weight. */
int64_t wo_fixed_from_f32(float w, int frac_bits)
{
    return (int64_t)rint(ldexp((double)w, frac_bits));
}

void wo_fixed_from_f32_array(const float *w, int64_t n, int frac_bits, int64_t *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = wo_fixed_from_f32(w[i], frac_bits);
}

/* Scatter-add of Section 2 ("Tensor Operations", item 7, Eq. "difftensor"):
 * S[i][I[i][k]] += V[k] for i < m0, k < m2.  S is [m0][m1], I is [m0][m2]. */
void wo_scatter_add(int64_t m0, int64_t m1, int64_t m2, const int64_t *I, const int64_t *V, int64_t *S)
{
    for (int64_t i = 0; i < m0; ++i)
        for (int64_t k = 0; k < m2; ++k) S[i * m1 + I[i * m2 + k]] += V[k];
}

/* Cumulative sum along the second axis (Section 2, item 4). */
void wo_cumsum_rows(int64_t m0, int64_t m1, int64_t *S)
{
    for (int64_t i = 0; i < m0; ++i)
        for (int64_t j = 1; j < m1; ++j) S[i * m1 + j] += S[i * m1 + j - 1];
}

/* Reduce-max along the second axis of an [m0][m1] table (Section 2, item 5). */
void wo_rmax_rows(int64_t m0, int64_t m1, const int64_t *T_, int64_t *out)
{
    for (int64_t i = 0; i < m0; ++i) {
        int64_t m = T_[i * m1];
        for (int64_t j = 1; j < m1; ++j)
            if (T_[i * m1 + j] > m) m = T_[i * m1 + j];
        out[i] = m;
    }
}

static int popcount_u(unsigned x)
{
    int c = 0;
    while (x) { c += (int)(x & 1u); x >>= 1; }
    return c;
}

/* ---------------------------------------------------------------- simplicial */

/*
 * Per-simplex weights as the maximum of the vertex weights (the Figure 1 convention).
 * simplices: [k][dim+1] vertex ids; out: [k].
 */
void wo_simplex_weights_max(int dim, int64_t k, const int32_t *simplices, const int64_t *vw, int64_t *out)
{
    for (int64_t b = 0; b < k; ++b) {
        int64_t m = vw[simplices[b * (dim + 1)]];
        for (int j = 1; j <= dim; ++j) {
            int64_t w = vw[simplices[b * (dim + 1) + j]];
            if (w > m) m = w;
        }
        out[b] = m;
    }
}

/* Largest |h_p(v)| over all directions and vertices: the M of Section 3. */
double wo_max_abs_height(int n, int64_t nv, const double *coords, int d, const double *dirs)
{
    double M = 0.0;
    for (int p = 0; p < d; ++p)
        for (int64_t v = 0; v < nv; ++v) {
            double h = fabs(wo_height(n, coords + v * n, dirs + (int64_t)p * n));
            if (h > M) M = h;
        }
    return M;
}

/*
 * Algorithm 1 (ComputeWECFs) for m = d filters given as a table f[p][v] (float64).
 * counts[0] = number of vertices; simplices[i] (i >= 1) is [counts[i]][i+1];
 * weights[i] is [counts[i]] int64 (weights[0] = vertex weights).
 * out: [d][T] int64.
 */
int wo_wecf_filters(int d, int64_t nv, const double *f, int max_dim, const int64_t *counts,
                    const int32_t *const *simplices, const int64_t *const *weights,
                    int T, double lo, double hi, int64_t *out)
{
    if (T < 2 || !(lo <= hi)) return WO_ERR;
    double *beta = (double *)malloc(sizeof(double) * (size_t)T);
    if (!beta) return WO_ERR;
    wo_beta(T, lo, hi, beta);
    for (int p = 0; p < d; ++p) {
        const double *fp = f + (int64_t)p * nv;
        int64_t *diff = out + (int64_t)p * T;
        for (int q = 0; q < T; ++q) diff[q] = 0;
        for (int i = 0; i <= max_dim; ++i) {
            int64_t sign = (i % 2 == 0) ? 1 : -1;
            for (int64_t b = 0; b < counts[i]; ++b) {
                double fmax;
                if (i == 0) {
                    fmax = fp[b];
                } else {
                    const int32_t *sv = simplices[i] + b * (i + 1);
                    fmax = fp[sv[0]];
                    for (int j = 1; j <= i; ++j)
                        if (fp[sv[j]] > fmax) fmax = fp[sv[j]];
                }
                diff[wo_bin(fmax, beta, T)] += sign * weights[i][b];
            }
        }
    }
    wo_cumsum_rows(d, T, out);
    free(beta);
    return WO_OK;
}

/* The WECT of a geometric simplicial complex (Example "ex:wect"): filters = heights. */
int wo_wect_simplicial(int n, int64_t nv, const double *coords, int max_dim, const int64_t *counts,
                       const int32_t *const *simplices, const int64_t *const *weights,
                       int d, const double *dirs, int T, double lo, double hi, int64_t *out)
{
    double *f = (double *)malloc(sizeof(double) * (size_t)nv * (size_t)(d > 0 ? d : 1));
    if (!f) return WO_ERR;
    for (int p = 0; p < d; ++p)
        for (int64_t v = 0; v < nv; ++v) f[(int64_t)p * nv + v] = wo_height(n, coords + v * n, dirs + (int64_t)p * n);
    int rc = wo_wecf_filters(d, nv, f, max_dim, counts, simplices, weights, T, lo, hi, out);
    free(f);
    return rc;
}

/* ---------------------------------------------------------------- cubical */

/* Flat index of a multi-index (axis 0 fastest). */
static int64_t flat_index(int n, const int64_t *dims, const int64_t *idx)
{
    int64_t v = 0;
    for (int a = n - 1; a >= 0; --a) v = v * dims[a] + idx[a];
    return v;
}

static int next_multi_index(int n, const int64_t *dims, int64_t *idx)
{
    for (int a = 0; a < n; ++a) {
        if (++idx[a] < dims[a]) return 1;
        idx[a] = 0;
    }
    return 0;
}

/*
 * WECF of the full cubical complex of an n-dimensional grid for d vertex filters f[p][v].
 * Cells are boxes (corner c, extent mask e) with c_a + e_a <= L_a - 1, of dimension
 * popcount(e).  Cell weight = max of its vertex weights (weighted != 0) or 1.
 */
int wo_wecf_cubical_filters(int n, const int64_t *dims, const int64_t *vw, int weighted,
                            int d, const double *f, int T, double lo, double hi, int64_t *out)
{
    if (n < 1 || n > 4 || T < 2 || !(lo <= hi)) return WO_ERR;
    int64_t nv = 1;
    for (int a = 0; a < n; ++a) {
        if (dims[a] < 1) return WO_ERR;
        nv *= dims[a];
    }
    double *beta = (double *)malloc(sizeof(double) * (size_t)T);
    if (!beta) return WO_ERR;
    wo_beta(T, lo, hi, beta);
    for (int p = 0; p < d; ++p) {
        const double *fp = f + (int64_t)p * nv;
        int64_t *diff = out + (int64_t)p * T;
        for (int q = 0; q < T; ++q) diff[q] = 0;
        int64_t c[4] = {0, 0, 0, 0};
        do {
            for (unsigned e = 0; e < (1u << n); ++e) {
                int fits = 1;
                for (int a = 0; a < n; ++a)
                    if (((e >> a) & 1u) && c[a] + 1 > dims[a] - 1) fits = 0;
                if (!fits) continue;
                double fmax = -INFINITY;
                int64_t wmax = INT64_MIN;
                /* every vertex of the box: corner + sub-mask of e */
                for (unsigned s = 0; s < (1u << n); ++s) {
                    if ((s & ~e) != 0) continue;
                    int64_t u[4];
                    for (int a = 0; a < n; ++a) u[a] = c[a] + (int64_t)((s >> a) & 1u);
                    int64_t v = flat_index(n, dims, u);
                    if (fp[v] > fmax) fmax = fp[v];
                    if (vw[v] > wmax) wmax = vw[v];
                }
                int64_t w = weighted ? wmax : 1;
                int64_t sign = (popcount_u(e) % 2 == 0) ? 1 : -1;
                diff[wo_bin(fmax, beta, T)] += sign * w;
            }
        } while (next_multi_index(n, dims, c));
    }
    wo_cumsum_rows(d, T, out);
    free(beta);
    return WO_OK;
}

/* Heights of every grid vertex for direction s. */
static void grid_heights(int n, const int64_t *dims, const double *s, double *h)
{
    int64_t idx[4] = {0, 0, 0, 0};
    double x[4];
    do {
        for (int a = 0; a < n; ++a) x[a] = wo_grid_coord(idx[a], dims[a]);
        h[flat_index(n, dims, idx)] = wo_height(n, x, s);
    } while (next_multi_index(n, dims, idx));
}

int wo_wect_cubical(int n, const int64_t *dims, const int64_t *vw, int weighted,
                    int d, const double *dirs, int T, double lo, double hi, int64_t *out)
{
    if (n < 1 || n > 4) return WO_ERR;
    int64_t nv = 1;
    for (int a = 0; a < n; ++a) nv *= dims[a];
    double *f = (double *)malloc(sizeof(double) * (size_t)nv);
    if (!f) return WO_ERR;
    for (int p = 0; p < d; ++p) {
        grid_heights(n, dims, dirs + (int64_t)p * n, f);
        int rc = wo_wecf_cubical_filters(n, dims, vw, weighted, 1, f, T, lo, hi, out + (int64_t)p * T);
        if (rc != WO_OK) { free(f); return rc; }
    }
    free(f);
    return WO_OK;
}

double wo_grid_max_abs_height(int n, const int64_t *dims, int d, const double *dirs)
{
    int64_t nv = 1;
    for (int a = 0; a < n; ++a) nv *= dims[a];
    double *h = (double *)malloc(sizeof(double) * (size_t)nv);
    if (!h) return NAN;
    double M = 0.0;
    for (int p = 0; p < d; ++p) {
        grid_heights(n, dims, dirs + (int64_t)p * n, h);
        for (int64_t v = 0; v < nv; ++v)
            if (fabs(h[v]) > M) M = fabs(h[v]);
    }
    free(h);
    return M;
}

/* ---------------------------------------------------------------- adjoint */

/*
 * Exact adjoint of the weighted transform with respect to the vertex weights, for
 * simplex weights that are the maximum of their vertex weights.  The paper leaves
 * differentiation to future work (Section 6); this is its plain chain rule:
 *   dW[p][q] / dw(s) = (-1)^dim(s) [bin_p(s) <= q],   dw(s)/dw_v = [v = argmax of s],
 * so with S[p][q] = sum_{q' >= q} G[p][q'] (the suffix sum of the upstream G),
 *   I_v = sum over simplices s whose heaviest vertex is v of (-1)^dim(s) sum_p S[p][bin_p(s)].
 * G is int64 (upstream gradient in fixed-point units); I_v is summed exactly in 128 bits;
 * grad[v] = (float)((double)I_v * scale).  Ties of the heaviest vertex go to the lowest index.
 */
static void suffix_sums(int d, int T, const int64_t *G, int64_t *S)
{
    for (int p = 0; p < d; ++p) {
        int64_t acc = 0;
        for (int q = T - 1; q >= 0; --q) {
            acc += G[(int64_t)p * T + q];
            S[(int64_t)p * T + q] = acc;
        }
    }
}

int wo_wect_backward_cubical(int n, const int64_t *dims, const int64_t *vw, int d, const double *dirs,
                             int T, double lo, double hi, const int64_t *G, double scale, float *grad)
{
    if (n < 1 || n > 4 || T < 2 || !(lo <= hi)) return WO_ERR;
    int64_t nv = 1;
    for (int a = 0; a < n; ++a) nv *= dims[a];
    double *beta = (double *)malloc(sizeof(double) * (size_t)T);
    double *h = (double *)malloc(sizeof(double) * (size_t)nv);
    int64_t *S = (int64_t *)malloc(sizeof(int64_t) * (size_t)d * (size_t)T);
    __int128 *I = (__int128 *)calloc((size_t)nv, sizeof(__int128));
    if (!beta || !h || !S || !I) { free(beta); free(h); free(S); free(I); return WO_ERR; }
    wo_beta(T, lo, hi, beta);
    suffix_sums(d, T, G, S);
    for (int p = 0; p < d; ++p) {
        grid_heights(n, dims, dirs + (int64_t)p * n, h);
        int64_t c[4] = {0, 0, 0, 0};
        do {
            for (unsigned e = 0; e < (1u << n); ++e) {
                int fits = 1;
                for (int a = 0; a < n; ++a)
                    if (((e >> a) & 1u) && c[a] + 1 > dims[a] - 1) fits = 0;
                if (!fits) continue;
                double hmax = -INFINITY;
                int64_t wmax = INT64_MIN, arg = -1;
                for (unsigned s = 0; s < (1u << n); ++s) {
                    if ((s & ~e) != 0) continue;
                    int64_t u[4];
                    for (int a = 0; a < n; ++a) u[a] = c[a] + (int64_t)((s >> a) & 1u);
                    int64_t v = flat_index(n, dims, u);
                    if (h[v] > hmax) hmax = h[v];
                    if (vw[v] > wmax || (vw[v] == wmax && v < arg)) { wmax = vw[v]; arg = v; }
                }
                int64_t sv = S[(int64_t)p * T + wo_bin(hmax, beta, T)];
                if (popcount_u(e) % 2 == 0) I[arg] += sv; else I[arg] -= sv;
            }
        } while (next_multi_index(n, dims, c));
    }
    for (int64_t v = 0; v < nv; ++v) grad[v] = (float)((double)I[v] * scale);
    free(beta); free(h); free(S); free(I);
    return WO_OK;
}

int wo_wect_backward_simplicial(int n, int64_t nv, const double *coords, const int64_t *vw, int max_dim,
                                const int64_t *counts, const int32_t *const *simplices,
                                int d, const double *dirs, int T, double lo, double hi,
                                const int64_t *G, double scale, float *grad)
{
    if (T < 2 || !(lo <= hi)) return WO_ERR;
    double *beta = (double *)malloc(sizeof(double) * (size_t)T);
    double *h = (double *)malloc(sizeof(double) * (size_t)nv);
    int64_t *S = (int64_t *)malloc(sizeof(int64_t) * (size_t)d * (size_t)T);
    __int128 *I = (__int128 *)calloc((size_t)nv, sizeof(__int128));
    if (!beta || !h || !S || !I) { free(beta); free(h); free(S); free(I); return WO_ERR; }
    wo_beta(T, lo, hi, beta);
    suffix_sums(d, T, G, S);
    for (int p = 0; p < d; ++p) {
        for (int64_t v = 0; v < nv; ++v) h[v] = wo_height(n, coords + v * n, dirs + (int64_t)p * n);
        for (int i = 0; i <= max_dim; ++i) {
            for (int64_t b = 0; b < counts[i]; ++b) {
                double hmax;
                int64_t arg;
                if (i == 0) {
                    hmax = h[b];
                    arg = b;
                } else {
                    const int32_t *sv = simplices[i] + b * (i + 1);
                    hmax = -INFINITY;
                    int64_t wmax = INT64_MIN;
                    arg = -1;
                    for (int j = 0; j <= i; ++j) {
                        int64_t v = sv[j];
                        if (h[v] > hmax) hmax = h[v];
                        if (vw[v] > wmax || (vw[v] == wmax && v < arg)) { wmax = vw[v]; arg = v; }
                    }
                }
                int64_t s = S[(int64_t)p * T + wo_bin(hmax, beta, T)];
                if (i % 2 == 0) I[arg] += s; else I[arg] -= s;
            }
        }
    }
    for (int64_t v = 0; v < nv; ++v) grad[v] = (float)((double)I[v] * scale);
    free(beta); free(h); free(S); free(I);
    return WO_OK;
}

/* 128-bit integer (hi, lo words) to the nearest double, for pinning the adjoint's last step. */
double wo_i128_to_double(int64_t hi, uint64_t lo)
{
    __int128 v = ((__int128)hi << 64) | (__int128)lo;
    return (double)v;
}
