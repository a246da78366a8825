/*
 * oracle.c -- plain, slow, FP64 CPU oracle for NSGA-III environmental
 * selection and the variation / objective around it.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this
 * file: it is loaded by tests/, by __graft_entry__.smoke() (to check one
 * small GPU call) and by bench.py's cpu_baseline / reference leg.  It shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * Every routine follows the paper's definitions step by step, in the
 * paper's order, with no blocking, fusion or reordering:
 *   - dominance and non-dominated sorting:  Sec. II-C, Alg. 1 (the
 *     non-dominated sort), minimisation as in Eq. (1);
 *   - reference directions: Sec. II-C (points uniform on the unit simplex,
 *     w close to n), Das-Dennis lattice;
 *   - normalization: the normalization step of Alg. 1 and Alg. 2;
 *     the paper gives no formula, so the Deb & Jain (NSGA-III) reading is
 *     used: ideal point, ASF extreme points, hyperplane intercepts;
 *   - perpendicular distance and association: Eq. (2) (read with cos^2,
 *     i.e. the true perpendicular distance of Fig. 1) and Alg. 2 argmin/min;
 *   - niche selection: Alg. 1 while-loop (primary) and the cached batched
 *     loop of Alg. 2 with truncation of the last batch (cross-check);
 *   - variation: binary tournament, SBX and polynomial mutation (Sec. II-C,
 *     Sec. III-A), standard bounded forms;
 *   - randomness: Philox4x32-10 (Salmon et al., SC'11) with counter
 *     (index, generation, stream, word3) and key (seed lo, seed hi).
 *
 * Compile with -ffp-contract=off (no FMA contraction) and without
 * -ffast-math: every FP64 operation is a separately rounded IEEE operation
 * in the order written.
 *
 * With -fopenmp the loops whose iterations are independent -- the
 * dominator count and the per-front sweep of the non-dominated sort (one
 * iteration per member j) and the association (one iteration per member
 * i) -- run on all host cores.  Each iteration does exactly the serial
 * arithmetic and writes only its own outputs, so the results are the same
 * bit for bit with any number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* ---------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as */
/* easy as 1, 2, 3", SC'11).  Round: two 32x32->64 multiplies by the      */
/* published multipliers, outputs permuted and xor-ed with the round key;  */
/* the key is bumped by the published Weyl constants between rounds.      */
/* ---------------------------------------------------------------------- */
static void orc_mulhilo(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)(p & 0xffffffffu);
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0, lo0, hi1, lo1;
        orc_mulhilo(0xD2511F53u, x0, &hi0, &lo0);
        orc_mulhilo(0xCD9E8D57u, x2, &hi1, &lo1);
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One Philox block for (index, gen, stream, word3) under seed. */
static void orc_draw(uint64_t seed, uint32_t index, uint32_t gen, uint32_t stream,
                     uint32_t word3, uint32_t out[4])
{
    uint32_t ctr[4] = {index, gen, stream, word3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Uniform in [0,1): top 24 bits of a word times 2^-24 (exact in float). */
static double orc_uniform(uint32_t w)
{
    return (double)(w >> 8) * (1.0 / 16777216.0);
}

/* Integer in [0, n): (w * n) >> 32. */
static uint32_t orc_bounded(uint32_t w, uint32_t n)
{
    return (uint32_t)(((uint64_t)w * (uint64_t)n) >> 32);
}

/* Random-number streams (third counter word). */
enum {
    ORC_STREAM_TOURNAMENT = 1,
    ORC_STREAM_SBX = 2,
    ORC_STREAM_PM = 3,
    ORC_STREAM_REFPRIO = 4,
    ORC_STREAM_MEMPRIO = 5,
    ORC_STREAM_INIT = 6
};

uint32_t orc_ref_priority(uint64_t seed, uint32_t gen, uint32_t j)
{
    uint32_t o[4];
    orc_draw(seed, j, gen, ORC_STREAM_REFPRIO, 0, o);
    return o[0];
}

uint32_t orc_member_priority(uint64_t seed, uint32_t gen, uint32_t i)
{
    uint32_t o[4];
    orc_draw(seed, i, gen, ORC_STREAM_MEMPRIO, 0, o);
    return o[0];
}

/* ---------------------------------------------------------------------- */
/* Reference directions: Das-Dennis lattice {k/p : k in N^m, sum k = p},   */
/* uniform on the unit simplex (Sec. II-C).  Order: lexicographic in       */
/* (k_0, ..., k_{m-1}) ascending.  Optional inner layer p2 shrunk toward   */
/* the centroid: z_in = (1 - tau)/m + tau * z.                             */
/* ---------------------------------------------------------------------- */
int64_t orc_binom(int n, int k)
{
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

int64_t orc_das_dennis_count(int m, int p)
{
    if (m < 1 || p < 0) return 0;
    return orc_binom(p + m - 1, m - 1);
}

static void orc_dd_rec(int m, int p, int q, int left, int *k, double *Z, int64_t *row,
                       int inner, double tau)
{
    if (q == m - 1) {
        k[q] = left;
        for (int r = 0; r < m; ++r) {
            double z = (double)k[r] / (double)p;
            if (inner) {
                double a = (1.0 - tau) / (double)m;
                double b = tau * z;
                z = a + b;
            }
            Z[(*row) * m + r] = z;
        }
        (*row)++;
        return;
    }
    for (int v = 0; v <= left; ++v) {
        k[q] = v;
        orc_dd_rec(m, p, q + 1, left - v, k, Z, row, inner, tau);
    }
}

/* Writes w x m directions (outer layer then inner layer); returns w. */
int64_t orc_refdirs(int m, int p1, int p2, double tau, double *Z)
{
    if (m < 2 || p1 < 1 || p2 < 0) return -1;
    int *k = (int *)malloc((size_t)m * sizeof(int));
    if (!k) return -1;
    int64_t row = 0;
    orc_dd_rec(m, p1, 0, p1, k, Z, &row, 0, tau);
    if (p2 > 0) orc_dd_rec(m, p2, 0, p2, k, Z, &row, 1, tau);
    free(k);
    return row;
}

/* ---------------------------------------------------------------------- */
/* Dominance (minimisation, Eq. 1): a dominates b iff a_q <= b_q for all q */
/* and a_q < b_q for some q.  Values are FP32 widened exactly to FP64.     */
/* ---------------------------------------------------------------------- */
int orc_dominates(const float *a, const float *b, int m)
{
    int all_le = 1, any_lt = 0;
    for (int q = 0; q < m; ++q) {
        double x = (double)a[q], y = (double)b[q];
        if (!(x <= y)) all_le = 0;
        if (x < y) any_lt = 1;
    }
    return all_le && any_lt;
}

/* ---------------------------------------------------------------------- */
/* Non-dominated sorting (Sec. II-C, Alg. 1).  F_1 = members of R not      */
/* dominated by any member of R; F_{k+1} the same on R minus F_1..F_k.     */
/* Realised by dominator counting: a member enters the next front when     */
/* its count of not-yet-ranked dominators reaches 0.  Sorting stops after  */
/* the first front l with |F_1|+...+|F_l| >= N (Alg. 1: F_s, F_l, F_drop); */
/* full_sort goes on ranking every member (l is still that first front).   */
/* rank = 0-based front index, -1 = F_drop.  Returns l, or -1 on error.    */
/* ---------------------------------------------------------------------- */
int orc_nds(const float *F, int n2, int m, int N, int full_sort, int32_t *rank)
{
    int *cnt = (int *)calloc((size_t)n2 > 0 ? (size_t)n2 : 1, sizeof(int));
    int *front = (int *)malloc(((size_t)n2 > 0 ? (size_t)n2 : 1) * sizeof(int));
    if (!cnt || !front) { free(cnt); free(front); return -1; }
    for (int j = 0; j < n2; ++j) rank[j] = -1;
    /* dominator count of every member j */
#pragma omp parallel for schedule(dynamic, 64)
    for (int j = 0; j < n2; ++j) {
        int c = 0;
        for (int i = 0; i < n2; ++i)
            if (orc_dominates(F + (size_t)i * m, F + (size_t)j * m, m)) c++;
        cnt[j] = c;
    }
    int nf = 0;
    for (int j = 0; j < n2; ++j)
        if (cnt[j] == 0) front[nf++] = j;
    int k = 0, cum = 0, l = -1;
    while (nf > 0) {
        for (int t = 0; t < nf; ++t) rank[front[t]] = k;
        cum += nf;
        if (l < 0 && cum >= N) l = k;
        if (!full_sort && cum >= N) break;
        /* every unranked member loses the dominators that front k held */
#pragma omp parallel for schedule(dynamic, 64)
        for (int j = 0; j < n2; ++j) {
            if (rank[j] != -1) continue;
            for (int t = 0; t < nf; ++t)
                if (orc_dominates(F + (size_t)front[t] * m, F + (size_t)j * m, m)) cnt[j]--;
        }
        /* the next front: unranked members left with no dominator, in
           ascending index order */
        int nn = 0;
        for (int j = 0; j < n2; ++j)
            if (rank[j] == -1 && cnt[j] == 0) front[nn++] = j;
        nf = nn;
        ++k;
    }
    free(cnt); free(front);
    return l;
}

/* Host threads the parallel loops use (1 without OpenMP). */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Normalization (the normalization step of Alg. 1 and Alg. 2).           */
/* Reading (Deb & Jain NSGA-III, stateless, current generation only):      */
/*   T = S u F_l (rank in [0, l]);                                         */
/*   ideal  z*_q = min_{i in T} f_iq;  translated ft_iq = f_iq - z*_q;     */
/*   extreme e_q = argmin_{i in T} max_r ft_ir / w_qr, w_qr = 1 (r == q),  */
/*                 1e-6 otherwise; ties -> lowest index;                   */
/*   solve E b = 1 (rows of E = ft at the extremes) by Gaussian            */
/*   elimination with partial pivoting (first maximal |pivot|); back       */
/*   substitution subtracts the known terms of a row from the highest      */
/*   column down: b_r = (rhs_r - A_r,m-1 b_m-1 - ... - A_r,r+1 b_r+1)/A_rr; */
/*   intercept a_q = 1 / b_q;                                              */
/*   fallback when a pivot is 0, an a_q is not finite or a_q <= 1e-6:      */
/*   a_q = max_{i in T} ft_iq for every q, and 1 where that is 0.          */
/* Outputs zstar[m], a[m], extremes[m]; *fallback = 1 if used.             */
/* ---------------------------------------------------------------------- */
/* element (i, j) of the row-major m x m system / extreme vectors */
#define AQ(i, j) A[(size_t)(i) * m + (j)]
#define EV(i, j) evec[(size_t)(i) * m + (j)]

int orc_normalize(const float *F, const int32_t *rank, int n2, int m, int l,
                  double *zstar, double *a, int32_t *extremes, int32_t *fallback)
{
    for (int q = 0; q < m; ++q) zstar[q] = INFINITY;
    int any = 0;
    for (int i = 0; i < n2; ++i) {
        if (rank[i] < 0 || rank[i] > l) continue;
        any = 1;
        for (int q = 0; q < m; ++q) {
            double v = (double)F[(size_t)i * m + q];
            if (v < zstar[q]) zstar[q] = v;
        }
    }
    if (!any) return ORC_EINVAL;
    /* -0.0 and +0.0 are the same minimum; keep +0.0 so that f - z* is defined
       by the value alone */
    for (int q = 0; q < m; ++q) zstar[q] = zstar[q] + 0.0;

    /* ASF extreme points */
    for (int q = 0; q < m; ++q) {
        double best = INFINITY;
        int32_t arg = -1;
        for (int i = 0; i < n2; ++i) {
            if (rank[i] < 0 || rank[i] > l) continue;
            double asf = -INFINITY;
            for (int r = 0; r < m; ++r) {
                double ft = (double)F[(size_t)i * m + r] - zstar[r];
                double wq = (r == q) ? 1.0 : 1e-6;
                double v = ft / wq;
                if (v > asf) asf = v;
            }
            if (asf < best) { best = asf; arg = i; }
        }
        extremes[q] = arg;
    }

    /* Gaussian elimination with partial pivoting on E b = 1 */
    double *A = (double *)malloc((size_t)m * m * sizeof(double));
    double *rhs = (double *)malloc((size_t)m * sizeof(double));
    double *b = (double *)malloc((size_t)m * sizeof(double));
    if (!A || !rhs || !b) { free(A); free(rhs); free(b); return ORC_ENOMEM; }
    for (int q = 0; q < m; ++q) {
        for (int r = 0; r < m; ++r)
            AQ(q, r) = (double)F[(size_t)extremes[q] * m + r] - zstar[r];
        rhs[q] = 1.0;
    }
    int ok = 1;
    for (int c = 0; c < m && ok; ++c) {
        int p = c;
        double best = fabs(AQ(c, c));
        for (int r = c + 1; r < m; ++r)
            if (fabs(AQ(r, c)) > best) { best = fabs(AQ(r, c)); p = r; }
        if (best == 0.0) { ok = 0; break; }
        if (p != c) {
            for (int cc = 0; cc < m; ++cc) { double t = AQ(c, cc); AQ(c, cc) = AQ(p, cc); AQ(p, cc) = t; }
            double t = rhs[c]; rhs[c] = rhs[p]; rhs[p] = t;
        }
        for (int r = c + 1; r < m; ++r) {
            double factor = AQ(r, c) / AQ(c, c);
            for (int cc = c; cc < m; ++cc) {
                double prod = factor * AQ(c, cc);
                AQ(r, cc) = AQ(r, cc) - prod;
            }
            double prod = factor * rhs[c];
            rhs[r] = rhs[r] - prod;
        }
    }
    if (ok) {
        for (int r = m - 1; r >= 0; --r) {
            double s = rhs[r];
            for (int cc = m - 1; cc > r; --cc) {
                double prod = AQ(r, cc) * b[cc];
                s = s - prod;
            }
            b[r] = s / AQ(r, r);
        }
        for (int q = 0; q < m; ++q) {
            a[q] = 1.0 / b[q];
            if (!isfinite(a[q]) || a[q] <= 1e-6) ok = 0;
        }
    }
    *fallback = ok ? 0 : 1;
    if (!ok) {
        for (int q = 0; q < m; ++q) {
            double mx = 0.0;
            for (int i = 0; i < n2; ++i) {
                if (rank[i] < 0 || rank[i] > l) continue;
                double ft = (double)F[(size_t)i * m + q] - zstar[q];
                if (ft > mx) mx = ft;
            }
            a[q] = (mx == 0.0) ? 1.0 : mx;
        }
    }
    free(A); free(rhs); free(b);
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Normalization with history (an option; the paper defines no history,   */
/* so this is the reading of a running ideal point and remembered extreme */
/* points, as several NSGA-III implementations keep them):                */
/*   z*_q = min(previous z*_q, min over ALL 2N merged points of f_q);     */
/*   extreme candidates: the members of T = S u F_l in index order, then  */
/*   the m remembered extreme vectors (candidate index 2N + r), ASF       */
/*   argmin per axis as in orc_normalize (ties -> lowest index);          */
/*   E b = 1 with the candidates' vectors, same elimination and fallback  */
/*   (the nadir fallback still maximises over T);                         */
/*   afterwards z* and the chosen extreme vectors become the history.     */
/* The history (hvalid, hz[m], he[m*m] FP32 vectors) is updated only when */
/* a normalization is computed.                                           */
/* ---------------------------------------------------------------------- */
int orc_normalize_hist(const float *F, const int32_t *rank, int n2, int m, int l, int32_t *hvalid,
                       double *hz, float *he, double *zstar, double *a, int32_t *extremes,
                       int32_t *fallback)
{
    for (int q = 0; q < m; ++q) zstar[q] = *hvalid ? hz[q] : INFINITY;
    int any = 0;
    for (int i = 0; i < n2; ++i) {
        if (rank[i] >= 0 && rank[i] <= l) any = 1;
        for (int q = 0; q < m; ++q) {
            double v = (double)F[(size_t)i * m + q];
            if (v < zstar[q]) zstar[q] = v;
        }
    }
    if (!any) return ORC_EINVAL;
    for (int q = 0; q < m; ++q) zstar[q] = zstar[q] + 0.0;

    /* candidate c: c < n2 -> row c of F (members of T only), c >= n2 ->
       remembered vector c - n2 */
    const int ncand = n2 + (*hvalid ? m : 0);
    for (int q = 0; q < m; ++q) {
        double best = INFINITY;
        int32_t arg = -1;
        for (int c = 0; c < ncand; ++c) {
            const float *f;
            if (c < n2) {
                if (rank[c] < 0 || rank[c] > l) continue;
                f = F + (size_t)c * m;
            } else {
                f = he + (size_t)(c - n2) * m;
            }
            double asf = -INFINITY;
            for (int r = 0; r < m; ++r) {
                double ft = (double)f[r] - zstar[r];
                double wq = (r == q) ? 1.0 : 1e-6;
                double v = ft / wq;
                if (v > asf) asf = v;
            }
            if (asf < best) { best = asf; arg = c; }
        }
        extremes[q] = arg;
    }
    float *evec = (float *)malloc((size_t)m * m * sizeof(float));
    if (!evec) return ORC_ENOMEM;
    for (int q = 0; q < m; ++q) {
        const float *f = extremes[q] < n2 ? F + (size_t)extremes[q] * m : he + (size_t)(extremes[q] - n2) * m;
        for (int r = 0; r < m; ++r) EV(q, r) = f[r];
    }

    double *A = (double *)malloc((size_t)m * m * sizeof(double));
    double *rhs = (double *)malloc((size_t)m * sizeof(double));
    double *b = (double *)malloc((size_t)m * sizeof(double));
    if (!A || !rhs || !b) { free(A); free(rhs); free(b); free(evec); return ORC_ENOMEM; }
    for (int q = 0; q < m; ++q) {
        for (int r = 0; r < m; ++r) AQ(q, r) = (double)EV(q, r) - zstar[r];
        rhs[q] = 1.0;
    }
    int ok = 1;
    for (int c = 0; c < m && ok; ++c) {
        int p = c;
        double best = fabs(AQ(c, c));
        for (int r = c + 1; r < m; ++r)
            if (fabs(AQ(r, c)) > best) { best = fabs(AQ(r, c)); p = r; }
        if (best == 0.0) { ok = 0; break; }
        if (p != c) {
            for (int cc = 0; cc < m; ++cc) { double t = AQ(c, cc); AQ(c, cc) = AQ(p, cc); AQ(p, cc) = t; }
            double t = rhs[c]; rhs[c] = rhs[p]; rhs[p] = t;
        }
        for (int r = c + 1; r < m; ++r) {
            double factor = AQ(r, c) / AQ(c, c);
            for (int cc = c; cc < m; ++cc) {
                double prod = factor * AQ(c, cc);
                AQ(r, cc) = AQ(r, cc) - prod;
            }
            double prod = factor * rhs[c];
            rhs[r] = rhs[r] - prod;
        }
    }
    if (ok) {
        for (int r = m - 1; r >= 0; --r) {
            double sum = rhs[r];
            for (int cc = m - 1; cc > r; --cc) {
                double prod = AQ(r, cc) * b[cc];
                sum = sum - prod;
            }
            b[r] = sum / AQ(r, r);
        }
        for (int q = 0; q < m; ++q) {
            a[q] = 1.0 / b[q];
            if (!isfinite(a[q]) || a[q] <= 1e-6) ok = 0;
        }
    }
    *fallback = ok ? 0 : 1;
    if (!ok) {
        for (int q = 0; q < m; ++q) {
            double mx = 0.0;
            for (int i = 0; i < n2; ++i) {
                if (rank[i] < 0 || rank[i] > l) continue;
                double ft = (double)F[(size_t)i * m + q] - zstar[q];
                if (ft > mx) mx = ft;
            }
            a[q] = (mx == 0.0) ? 1.0 : mx;
        }
    }
    for (int q = 0; q < m; ++q) {
        hz[q] = zstar[q];
        for (int r = 0; r < m; ++r) he[(size_t)q * m + r] = EV(q, r);
    }
    *hvalid = 1;
    free(A); free(rhs); free(b); free(evec);
    return ORC_OK;
}

#undef AQ
#undef EV

/* ---------------------------------------------------------------------- */
/* Association (Alg. 2: perpendicular distances, pi = argmin, d = min;     */
/* Eq. 2 read as D = |F| * sqrt(1 - cos^2), cos = F.Z / (|F||Z|)).         */
/* For i in T: f'_q = (f_iq - z*_q) / a_q;  nf = sqrt(sum f'_q^2);          */
/* nz_j = sqrt(sum z_jq^2);  dot = sum f'_q z_jq;  c = dot / (nf * nz_j);  */
/* D_ij = nf * sqrt(max(0, 1 - c*c));  nf == 0 -> D_ij = 0 for all j.     */
/* Sums run left to right over q.  pi_i = first j of minimal D_ij.         */
/* Members outside T get pi = -1, d = 0.                                   */
/* ---------------------------------------------------------------------- */
void orc_associate(const float *F, const int32_t *rank, int n2, int m, int l,
                   const double *zstar, const double *a, const double *Z, int w,
                   int32_t *pi, double *dist)
{
    double *nz = (double *)malloc((size_t)(w > 0 ? w : 1) * sizeof(double));
    for (int j = 0; j < w; ++j) {
        double s = 0.0;
        for (int q = 0; q < m; ++q) {
            double sq = Z[(size_t)j * m + q] * Z[(size_t)j * m + q];
            s = s + sq;
        }
        nz[j] = sqrt(s);
    }
#pragma omp parallel
    {
        double *fp = (double *)malloc((size_t)m * sizeof(double));
#pragma omp for schedule(dynamic, 16)
        for (int i = 0; i < n2; ++i) {
            pi[i] = -1;
            dist[i] = 0.0;
            if (rank[i] < 0 || rank[i] > l) continue;
            double s = 0.0;
            for (int q = 0; q < m; ++q) {
                double ft = (double)F[(size_t)i * m + q] - zstar[q];
                fp[q] = ft / a[q];
                double sq = fp[q] * fp[q];
                s = s + sq;
            }
            double nf = sqrt(s);
            double best = INFINITY;
            int32_t arg = -1;
            for (int j = 0; j < w; ++j) {
                double D;
                if (nf == 0.0) {
                    D = 0.0;
                } else {
                    double dot = 0.0;
                    for (int q = 0; q < m; ++q) {
                        double pr = fp[q] * Z[(size_t)j * m + q];
                        dot = dot + pr;
                    }
                    double den = nf * nz[j];
                    double c = dot / den;
                    double cc = c * c;
                    double one_m = 1.0 - cc;
                    if (one_m < 0.0) one_m = 0.0;
                    D = nf * sqrt(one_m);
                }
                if (D < best) { best = D; arg = j; }
            }
            pi[i] = arg;
            dist[i] = best;
        }
        free(fp);
    }
    free(nz);
}

/* ---------------------------------------------------------------------- */
/* Niche selection.  Inputs: rank (l = selecting front), pi, dist; picks   */
/* K = N - |S| members of F_l.  Random choices are realised by fixed       */
/* Philox priorities of this generation: the random pick of a reference   */
/* among those of minimum niche count takes the one of smallest            */
/* (ref priority, j); the random pick of a member takes the remaining      */
/* member of smallest (member priority, i).  picked[i] = 1 for chosen i.   */
/* ---------------------------------------------------------------------- */

/* Alg. 1 while-loop, literally. */
int orc_niche_sequential(const int32_t *rank, int n2, int l, int K,
                         const int32_t *pi, const double *dist, int w,
                         uint64_t seed, uint32_t gen, uint8_t *picked)
{
    int *rho = (int *)calloc((size_t)w, sizeof(int));
    int *rhop = (int *)calloc((size_t)w, sizeof(int));
    uint8_t *active = (uint8_t *)malloc((size_t)w);
    uint32_t *rprio = (uint32_t *)malloc((size_t)w * sizeof(uint32_t));
    uint32_t *mprio = (uint32_t *)malloc((size_t)(n2 > 0 ? n2 : 1) * sizeof(uint32_t));
    if (!rho || !rhop || !active || !rprio || !mprio) return ORC_ENOMEM;
    for (int i = 0; i < n2; ++i) picked[i] = 0;
    for (int i = 0; i < n2; ++i) mprio[i] = orc_member_priority(seed, gen, (uint32_t)i);
    for (int i = 0; i < n2; ++i) {
        if (rank[i] >= 0 && rank[i] < l) rho[pi[i]]++;
        else if (rank[i] == l) rhop[pi[i]]++;
    }
    for (int j = 0; j < w; ++j) { active[j] = 1; rprio[j] = orc_ref_priority(seed, gen, (uint32_t)j); }
    int sel = 0;
    while (sel < K) {
        int v = -1;
        for (int j = 0; j < w; ++j) {
            if (!active[j]) continue;
            if (v < 0 || rho[j] < rho[v] ||
                (rho[j] == rho[v] && (rprio[j] < rprio[v] || (rprio[j] == rprio[v] && j < v))))
                v = j;
        }
        if (v < 0) break; /* cannot happen when K <= |F_l| */
        if (rhop[v] == 0) { active[v] = 0; continue; }
        int t = -1;
        if (rho[v] == 0) {
            for (int i = 0; i < n2; ++i) {
                if (rank[i] != l || picked[i] || pi[i] != v) continue;
                if (t < 0 || dist[i] < dist[t]) t = i;
            }
        } else {
            uint32_t bp = 0;
            for (int i = 0; i < n2; ++i) {
                if (rank[i] != l || picked[i] || pi[i] != v) continue;
                uint32_t pr = mprio[i];
                if (t < 0 || pr < bp) { t = i; bp = pr; }
            }
        }
        picked[t] = 1;
        sel++;
        rho[v]++;
        rhop[v]--;
    }
    free(rho); free(rhop); free(active); free(rprio); free(mprio);
    return sel == K ? ORC_OK : ORC_EINVAL;
}

/* Alg. 2 cached batched loop: nearest batch for rho == 0, then per-ref     */
/* queues Q (members in priority order) with cursor s; every iteration      */
/* takes one member from each ref of minimum count; the last batch is       */
/* truncated keeping refs in priority order (the shuffled-Z truncation).    */
typedef struct { int j; int i; } orc_pick;

static int orc_cmp_ref(const uint32_t *rprio, int a, int b)
{
    if (rprio[a] != rprio[b]) return rprio[a] < rprio[b] ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

static void orc_sort_batch(orc_pick *B, int nb, const uint32_t *rprio)
{
    for (int x = 1; x < nb; ++x) {
        orc_pick v = B[x];
        int y = x - 1;
        while (y >= 0 && orc_cmp_ref(rprio, B[y].j, v.j) > 0) { B[y + 1] = B[y]; --y; }
        B[y + 1] = v;
    }
}

int orc_niche_batched(const int32_t *rank, int n2, int l, int K,
                      const int32_t *pi, const double *dist, int w,
                      uint64_t seed, uint32_t gen, uint8_t *picked)
{
    const long INF = 1L << 40;
    long *rho = (long *)calloc((size_t)w, sizeof(long));
    int *rhop = (int *)calloc((size_t)w, sizeof(int));
    uint32_t *rprio = (uint32_t *)calloc((size_t)(w > 0 ? w : 1), sizeof(uint32_t));
    int *qoff = (int *)calloc((size_t)w + 1, sizeof(int));
    int *Q = (int *)malloc((size_t)(n2 > 0 ? n2 : 1) * sizeof(int));
    int *s = (int *)calloc((size_t)w, sizeof(int));
    orc_pick *B = (orc_pick *)malloc((size_t)(w > 0 ? w : 1) * sizeof(orc_pick));
    uint32_t *mprio = (uint32_t *)malloc((size_t)(n2 > 0 ? n2 : 1) * sizeof(uint32_t));
    if (!rho || !rhop || !rprio || !qoff || !Q || !s || !B || !mprio) return ORC_ENOMEM;
    for (int i = 0; i < n2; ++i) picked[i] = 0;
    for (int i = 0; i < n2; ++i) {
        mprio[i] = orc_member_priority(seed, gen, (uint32_t)i);
        if (rank[i] >= 0 && rank[i] < l) rho[pi[i]]++;
        else if (rank[i] == l) rhop[pi[i]]++;
    }
    for (int j = 0; j < w; ++j) {
        rprio[j] = orc_ref_priority(seed, gen, (uint32_t)j);
        if (rhop[j] == 0) rho[j] += INF; /* Alg. 2: rho += inf where rho' = 0 */
    }
    int sel = 0;
    /* nearest batch: refs with rho == 0 take their nearest member */
    int nb = 0;
    for (int j = 0; j < w; ++j) {
        if (rho[j] != 0) continue;
        int t = -1;
        for (int i = 0; i < n2; ++i) {
            if (rank[i] != l || pi[i] != j) continue;
            if (t < 0 || dist[i] < dist[t]) t = i;
        }
        B[nb].j = j; B[nb].i = t; nb++;
    }
    orc_sort_batch(B, nb, rprio);
    int keep = nb < K ? nb : K;
    for (int x = 0; x < keep; ++x) picked[B[x].i] = 1;
    sel += keep;
    for (int x = 0; x < nb; ++x) {
        int j = B[x].j;
        rhop[j] -= 1;
        rho[j] += 1;
        if (rhop[j] == 0) rho[j] += INF;
    }
    /* cache Q: per ref, its not-yet-picked F_l members in (priority, i) order */
    for (int i = 0; i < n2; ++i)
        if (rank[i] == l && !picked[i]) qoff[pi[i] + 1]++;
    for (int j = 0; j < w; ++j) qoff[j + 1] += qoff[j];
    int *fill = (int *)calloc((size_t)w, sizeof(int));
    for (int i = 0; i < n2; ++i)
        if (rank[i] == l && !picked[i]) Q[qoff[pi[i]] + fill[pi[i]]++] = i;
    free(fill);
    for (int j = 0; j < w; ++j) {
        int lo = qoff[j], hi = qoff[j + 1];
        for (int x = lo + 1; x < hi; ++x) {
            int v = Q[x], y = x - 1;
            while (y >= lo && (mprio[Q[y]] > mprio[v] || (mprio[Q[y]] == mprio[v] && Q[y] > v))) {
                Q[y + 1] = Q[y]; --y;
            }
            Q[y + 1] = v;
        }
    }
    while (sel < K) {
        long mn = INF;
        for (int j = 0; j < w; ++j) if (rho[j] < mn) mn = rho[j];
        if (mn >= INF) break;
        nb = 0;
        for (int j = 0; j < w; ++j) {
            if (rho[j] != mn) continue;
            B[nb].j = j; B[nb].i = Q[qoff[j] + s[j]]; nb++;
        }
        orc_sort_batch(B, nb, rprio);
        keep = nb < (K - sel) ? nb : (K - sel);
        for (int x = 0; x < keep; ++x) picked[B[x].i] = 1;
        sel += keep;
        for (int x = 0; x < nb; ++x) {
            int j = B[x].j;
            s[j] += 1;
            rhop[j] -= 1;
            rho[j] += 1;
            if (rhop[j] == 0) rho[j] += INF;
        }
    }
    free(rho); free(rhop); free(rprio); free(qoff); free(Q); free(s); free(B); free(mprio);
    return sel == K ? ORC_OK : ORC_EINVAL;
}

/* ---------------------------------------------------------------------- */
/* Full environmental selection over the merged 2N x m objectives:          */
/* sort, whole fronts into S, niche-select K = N - |S| from F_l, and return */
/* rank[2N] and selected[N] in ascending index order (the mask form of      */
/* Alg. 2's last line).  variant: 0 = Alg. 1 loop, 1 = Alg. 2 cached loop.  */
/* info[0..5] = l, |S|, K, |F_l|, niching used, normalization fallback.     */
/* ---------------------------------------------------------------------- */
int orc_select_hist(const float *F, int N, int m, const double *Z, int w, uint64_t seed,
                    uint32_t gen, int variant, int full_sort, int32_t *rank, int32_t *selected,
                    int32_t *pi_out, double *dist_out, int32_t *info, int32_t *hvalid,
                    double *hz, float *he);

int orc_select(const float *F, int N, int m, const double *Z, int w, uint64_t seed,
               uint32_t gen, int variant, int full_sort, int32_t *rank, int32_t *selected,
               int32_t *pi_out, double *dist_out, int32_t *info)
{
    return orc_select_hist(F, N, m, Z, w, seed, gen, variant, full_sort, rank, selected, pi_out,
                           dist_out, info, NULL, NULL, NULL);
}

/* As orc_select; with hvalid != NULL the normalization keeps a history   */
/* (orc_normalize_hist), else it is the stateless orc_normalize.          */
int orc_select_hist(const float *F, int N, int m, const double *Z, int w, uint64_t seed,
                    uint32_t gen, int variant, int full_sort, int32_t *rank, int32_t *selected,
                    int32_t *pi_out, double *dist_out, int32_t *info, int32_t *hvalid,
                    double *hz, float *he)
{
    int n2 = 2 * N;
    for (int i = 0; i < n2 * m; ++i)
        if (!isfinite((double)F[i])) return ORC_EINVAL;
    int l = orc_nds(F, n2, m, N, full_sort, rank);
    if (l < 0) return ORC_EINVAL;
    int nS = 0, nFl = 0;
    for (int i = 0; i < n2; ++i) {
        if (rank[i] >= 0 && rank[i] < l) nS++;
        else if (rank[i] == l) nFl++;
    }
    int K = N - nS;
    uint8_t *picked = (uint8_t *)calloc((size_t)n2, 1);
    int32_t *pi = (int32_t *)malloc((size_t)n2 * sizeof(int32_t));
    double *dist = (double *)malloc((size_t)n2 * sizeof(double));
    if (!picked || !pi || !dist) return ORC_ENOMEM;
    int niche = 0, fb = 0;
    for (int i = 0; i < n2; ++i) { pi[i] = -1; dist[i] = 0.0; }
    if (K == nFl) {
        for (int i = 0; i < n2; ++i) if (rank[i] == l) picked[i] = 1;
    } else {
        niche = 1;
        double *zstar = (double *)malloc((size_t)m * sizeof(double));
        double *a = (double *)malloc((size_t)m * sizeof(double));
        int32_t *ext = (int32_t *)malloc((size_t)m * sizeof(int32_t));
        if (!zstar || !a || !ext) return ORC_ENOMEM;
        if (hvalid)
            orc_normalize_hist(F, rank, n2, m, l, hvalid, hz, he, zstar, a, ext, &fb);
        else
            orc_normalize(F, rank, n2, m, l, zstar, a, ext, &fb);
        orc_associate(F, rank, n2, m, l, zstar, a, Z, w, pi, dist);
        free(zstar); free(a); free(ext);
        int rc = variant == 0
                     ? orc_niche_sequential(rank, n2, l, K, pi, dist, w, seed, gen, picked)
                     : orc_niche_batched(rank, n2, l, K, pi, dist, w, seed, gen, picked);
        if (rc != ORC_OK) return rc;
    }
    int c = 0;
    for (int i = 0; i < n2; ++i)
        if ((rank[i] >= 0 && rank[i] < l) || picked[i]) selected[c++] = i;
    if (pi_out) memcpy(pi_out, pi, (size_t)n2 * sizeof(int32_t));
    if (dist_out) memcpy(dist_out, dist, (size_t)n2 * sizeof(double));
    if (info) { info[0] = l; info[1] = nS; info[2] = K; info[3] = nFl; info[4] = niche; info[5] = fb; }
    free(picked); free(pi); free(dist);
    return c == N ? ORC_OK : ORC_EINVAL;
}

/* ---------------------------------------------------------------------- */
/* Variation (Sec. II-C: mating pool by tournament, SBX, polynomial         */
/* mutation; Sec. III-A).  For pair q in [0, N/2):                          */
/*   Philox(q, gen, 1, 0) -> a1, b1, a2, b2 uniform in [0, N); parent 1 =   */
/*   b1 if rank[b1] < rank[a1] else a1 (ties keep the first drawn); same    */
/*   for parent 2.  Philox(q, gen, 1, 1) word 0 < p_c -> the pair crosses.  */
/*   Per variable v: Philox(q*d + v, gen, 2, 0): word 1 < 0.5 -> SBX on v:  */
/*   u = word 0, beta = (2u)^(1/(eta_c+1)) if u <= 0.5 else                 */
/*   (1/(2(1-u)))^(1/(eta_c+1)); c1 = 0.5((1+beta)x1 + (1-beta)x2),         */
/*   c2 = 0.5((1-beta)x1 + (1+beta)x2); word 2 < 0.5 swaps c1, c2; clip.    */
/*   Children 2q, 2q+1.  Polynomial mutation (Deb & Goyal 1996, bounded     */
/*   form on [0,1]) of variable v: Philox(q*d + v, gen, 2, 0) word 3 < p_m  */
/*   mutates child 2q with u = word 0 of Philox(q*d + v, gen, 3, 0); word 1 */
/*   of that block < p_m mutates child 2q+1 with u = its word 2.            */
/* Probability tests compare the exact float uniform with the float        */
/* probability.  Arithmetic in FP64; children rounded to FP32.              */
/* ---------------------------------------------------------------------- */
void orc_vary(const float *X, const int32_t *rank, int N, int d, uint64_t seed, uint32_t gen,
              double eta_c, double eta_m, float p_c, float p_m, float *Xc)
{
    for (int q = 0; q < N / 2; ++q) {
        uint32_t t[4], cxw[4];
        orc_draw(seed, (uint32_t)q, gen, ORC_STREAM_TOURNAMENT, 0, t);
        orc_draw(seed, (uint32_t)q, gen, ORC_STREAM_TOURNAMENT, 1, cxw);
        uint32_t a1 = orc_bounded(t[0], (uint32_t)N), b1 = orc_bounded(t[1], (uint32_t)N);
        uint32_t a2 = orc_bounded(t[2], (uint32_t)N), b2 = orc_bounded(t[3], (uint32_t)N);
        uint32_t p1 = rank[b1] < rank[a1] ? b1 : a1;
        uint32_t p2 = rank[b2] < rank[a2] ? b2 : a2;
        int cross = (float)orc_uniform(cxw[0]) < p_c;
        for (int v = 0; v < d; ++v) {
            double x1 = (double)X[(size_t)p1 * d + v], x2 = (double)X[(size_t)p2 * d + v];
            double c1 = x1, c2 = x2;
            uint32_t s[4];
            orc_draw(seed, (uint32_t)q * (uint32_t)d + (uint32_t)v, gen, ORC_STREAM_SBX, 0, s);
            if (cross && (float)orc_uniform(s[1]) < 0.5f) {
                double u = orc_uniform(s[0]);
                double e = 1.0 / (eta_c + 1.0);
                double beta = (u <= 0.5) ? pow(2.0 * u, e) : pow(1.0 / (2.0 * (1.0 - u)), e);
                c1 = 0.5 * ((1.0 + beta) * x1 + (1.0 - beta) * x2);
                c2 = 0.5 * ((1.0 - beta) * x1 + (1.0 + beta) * x2);
                if ((float)orc_uniform(s[2]) < 0.5f) { double tt = c1; c1 = c2; c2 = tt; }
                if (c1 < 0.0) c1 = 0.0;
                if (c1 > 1.0) c1 = 1.0;
                if (c2 < 0.0) c2 = 0.0;
                if (c2 > 1.0) c2 = 1.0;
            }
            double ch[2] = {c1, c2};
            uint32_t pm[4];
            orc_draw(seed, (uint32_t)q * (uint32_t)d + (uint32_t)v, gen, ORC_STREAM_PM, 0, pm);
            const uint32_t pm_dec[2] = {s[3], pm[1]}, pm_u[2] = {pm[0], pm[2]};
            for (int h = 0; h < 2; ++h) {
                uint32_t c = 2u * (uint32_t)q + (uint32_t)h;
                double y = ch[h];
                if ((float)orc_uniform(pm_dec[h]) < p_m) {
                    double u = orc_uniform(pm_u[h]);
                    double d1 = y - 0.0, d2 = 1.0 - y;
                    double mp = 1.0 / (eta_m + 1.0);
                    double dq;
                    if (u < 0.5) {
                        double xy = 1.0 - d1;
                        double val = 2.0 * u + (1.0 - 2.0 * u) * pow(xy, eta_m + 1.0);
                        dq = pow(val, mp) - 1.0;
                    } else {
                        double xy = 1.0 - d2;
                        double val = 2.0 * (1.0 - u) + 2.0 * (u - 0.5) * pow(xy, eta_m + 1.0);
                        dq = 1.0 - pow(val, mp);
                    }
                    y = y + dq * (1.0 - 0.0);
                    if (y < 0.0) y = 0.0;
                    if (y > 1.0) y = 1.0;
                }
                Xc[(size_t)c * d + v] = (float)y;
            }
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Synthetic softmax-simplex objective (the stand-in problem family):      */
/* k = m - 1, g = sum_{v >= k} (x_v - 0.5)^2, s = softmax(W x[0:k]),        */
/* f_j = (1 + g) s_j.  On g = 0 the front satisfies sum f = 1.  FP64,       */
/* rounded to FP32.  W is m x k row-major.                                  */
/* ---------------------------------------------------------------------- */
void orc_eval(const float *X, int n, int d, int m, const float *W, float *F)
{
    int k = m - 1;
    double *e = (double *)malloc((size_t)m * sizeof(double));
    if (!e) return;
    for (int i = 0; i < n; ++i) {
        const float *x = X + (size_t)i * d;
        double g = 0.0;
        for (int v = k; v < d; ++v) {
            double t = (double)x[v] - 0.5;
            double sq = t * t;
            g = g + sq;
        }
        double den = 0.0;
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int v = 0; v < k; ++v) {
                double pr = (double)W[j * k + v] * (double)x[v];
                s = s + pr;
            }
            e[j] = exp(s);
            den = den + e[j];
        }
        for (int j = 0; j < m; ++j) {
            double sj = e[j] / den;
            F[(size_t)i * m + j] = (float)((1.0 + g) * sj);
        }
    }
    free(e);
}

/* x_iv = uniform(Philox(i*d + v, 0, 6, 0) word 0). */
void orc_init(int N, int d, uint64_t seed, float *X)
{
    for (int i = 0; i < N; ++i)
        for (int v = 0; v < d; ++v) {
            uint32_t o[4];
            orc_draw(seed, (uint32_t)i * (uint32_t)d + (uint32_t)v, 0, ORC_STREAM_INIT, 0, o);
            X[(size_t)i * d + v] = (float)orc_uniform(o[0]);
        }
}

/* ---------------------------------------------------------------------- */
/* One generation (Alg. 1): Q = vary(P); R = P u Q; select; P' = R[sel].   */
/* X, F, rank hold the N parents and are overwritten with the next ones.  */
/* ---------------------------------------------------------------------- */
int orc_generation(float *X, float *F, int32_t *rank, int N, int d, int m, const float *W,
                   const double *Z, int w, uint64_t seed, uint32_t gen, double eta_c,
                   double eta_m, float p_c, float p_m, int variant)
{
    int n2 = 2 * N;
    float *RX = (float *)malloc((size_t)n2 * d * sizeof(float));
    float *RF = (float *)malloc((size_t)n2 * m * sizeof(float));
    int32_t *rr = (int32_t *)malloc((size_t)n2 * sizeof(int32_t));
    int32_t *sel = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    if (!RX || !RF || !rr || !sel) return ORC_ENOMEM;
    memcpy(RX, X, (size_t)N * d * sizeof(float));
    memcpy(RF, F, (size_t)N * m * sizeof(float));
    orc_vary(X, rank, N, d, seed, gen, eta_c, eta_m, p_c, p_m, RX + (size_t)N * d);
    orc_eval(RX + (size_t)N * d, N, d, m, W, RF + (size_t)N * m);
    int rc = orc_select(RF, N, m, Z, w, seed, gen, variant, 0, rr, sel, NULL, NULL, NULL);
    if (rc == ORC_OK) {
        for (int p = 0; p < N; ++p) {
            memcpy(X + (size_t)p * d, RX + (size_t)sel[p] * d, (size_t)d * sizeof(float));
            memcpy(F + (size_t)p * m, RF + (size_t)sel[p] * m, (size_t)m * sizeof(float));
            rank[p] = rr[sel[p]];
        }
    }
    free(RX); free(RF); free(rr); free(sel);
    return rc;
}

/* ====================================================================== */
/* Second workload: 0-1 multi-objective knapsack, a reading of the         */
/* MOKnapsack family the paper evaluates (Sec. IV, App. E); the paper      */
/* gives no instance, so the instance data are inputs.  m knapsacks share */
/* d items with integer profits p[j][v] and weights w[j][v] > 0 and       */
/* capacities c[j].  Objectives (minimised, non-negative):                */
/*   f_j(x) = P_j - sum_v p[j][v] x_v,   P_j = sum_v p[j][v].             */
/* Repair to feasibility: items leave in a fixed order (ascending         */
/* max_j p[j][v] / w[j][v], ties to the lower item) while a knapsack      */
/* overflows; the repaired x replaces x.  All arithmetic is integer.      */
/* ====================================================================== */

/* 1 if item a's best profit/weight ratio is below item b's (exact, by    */
/* cross multiplication), ties broken by index. */
static int orc_kp_before(const int32_t *p, const int32_t *w, int m, int d, int a, int b)
{
    int64_t na = p[a], da = w[a], nb = p[b], db = w[b];
    for (int j = 1; j < m; ++j) {
        if ((int64_t)p[(size_t)j * d + a] * da > na * (int64_t)w[(size_t)j * d + a]) {
            na = p[(size_t)j * d + a];
            da = w[(size_t)j * d + a];
        }
        if ((int64_t)p[(size_t)j * d + b] * db > nb * (int64_t)w[(size_t)j * d + b]) {
            nb = p[(size_t)j * d + b];
            db = w[(size_t)j * d + b];
        }
    }
    if (na * db != nb * da) return na * db < nb * da;
    return a < b;
}

void orc_kp_order(const int32_t *p, const int32_t *w, int m, int d, int32_t *order)
{
    for (int v = 0; v < d; ++v) order[v] = v;
    for (int i = 1; i < d; ++i) {  /* insertion sort: plain and stable */
        int32_t x = order[i];
        int k = i - 1;
        while (k >= 0 && orc_kp_before(p, w, m, d, x, order[k])) {
            order[k + 1] = order[k];
            --k;
        }
        order[k + 1] = x;
    }
}

void orc_kp_eval(float *X, int n, int d, int m, const int32_t *p, const int32_t *w,
                 const int32_t *cap, const int32_t *order, float *F)
{
    int64_t *load = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    if (!load) return;
    for (int i = 0; i < n; ++i) {
        float *x = X + (size_t)i * d;
        for (int j = 0; j < m; ++j) {
            load[j] = 0;
            for (int v = 0; v < d; ++v)
                if (x[v] != 0.0f) load[j] += w[(size_t)j * d + v];
        }
        for (int k = 0; k < d; ++k) {
            int over = 0;
            for (int j = 0; j < m; ++j)
                if (load[j] > cap[j]) over = 1;
            if (!over) break;
            int v = order[k];
            if (x[v] != 0.0f) {
                x[v] = 0.0f;
                for (int j = 0; j < m; ++j) load[j] -= w[(size_t)j * d + v];
            }
        }
        for (int j = 0; j < m; ++j) {
            int64_t left = 0;
            for (int v = 0; v < d; ++v)
                if (x[v] == 0.0f) left += p[(size_t)j * d + v];
            F[(size_t)i * m + j] = (float)left;
        }
    }
    free(load);
}

/* Initial bits: Philox(i*d + v, 0, 6, 0) word 0 < 0.5 -> item v chosen.   */
void orc_kp_init(int N, int d, uint64_t seed, float *X)
{
    for (int i = 0; i < N; ++i)
        for (int v = 0; v < d; ++v) {
            uint32_t o[4];
            orc_draw(seed, (uint32_t)i * (uint32_t)d + (uint32_t)v, 0, ORC_STREAM_INIT, 0, o);
            X[(size_t)i * d + v] = ((float)orc_uniform(o[0]) < 0.5f) ? 1.0f : 0.0f;
        }
}

/* Binary variation: the tournament and crossover decision of orc_vary;   */
/* uniform crossover: Philox(q*d + v, gen, 2, 0) word 0 < 0.5 swaps the    */
/* parents' bits of item v between the children; bit-flip mutation:       */
/* Philox(q*d + v, gen, 3, 0) word 0 < p_m flips child 2q's bit, word 1   */
/* < p_m flips child 2q+1's bit.                                           */
void orc_kp_vary(const float *X, const int32_t *rank, int N, int d, uint64_t seed, uint32_t gen,
                 float p_c, float p_m, float *Xc)
{
    for (int q = 0; q < N / 2; ++q) {
        uint32_t t[4], cxw[4];
        orc_draw(seed, (uint32_t)q, gen, ORC_STREAM_TOURNAMENT, 0, t);
        orc_draw(seed, (uint32_t)q, gen, ORC_STREAM_TOURNAMENT, 1, cxw);
        uint32_t a1 = orc_bounded(t[0], (uint32_t)N), b1 = orc_bounded(t[1], (uint32_t)N);
        uint32_t a2 = orc_bounded(t[2], (uint32_t)N), b2 = orc_bounded(t[3], (uint32_t)N);
        uint32_t p1 = rank[b1] < rank[a1] ? b1 : a1;
        uint32_t p2 = rank[b2] < rank[a2] ? b2 : a2;
        int cross = (float)orc_uniform(cxw[0]) < p_c;
        for (int v = 0; v < d; ++v) {
            float c1 = X[(size_t)p1 * d + v], c2 = X[(size_t)p2 * d + v];
            uint32_t s[4], pm[4];
            orc_draw(seed, (uint32_t)q * (uint32_t)d + (uint32_t)v, gen, ORC_STREAM_SBX, 0, s);
            if (cross && (float)orc_uniform(s[0]) < 0.5f) { float tt = c1; c1 = c2; c2 = tt; }
            orc_draw(seed, (uint32_t)q * (uint32_t)d + (uint32_t)v, gen, ORC_STREAM_PM, 0, pm);
            if ((float)orc_uniform(pm[0]) < p_m) c1 = 1.0f - c1;
            if ((float)orc_uniform(pm[1]) < p_m) c2 = 1.0f - c2;
            Xc[(size_t)(2 * q) * d + v] = c1;
            Xc[(size_t)(2 * q + 1) * d + v] = c2;
        }
    }
}

/* One knapsack generation (Alg. 1): Q = vary(P), repaired and evaluated; */
/* R = P u Q; select; P' = R[sel].  X, F, rank are overwritten.           */
int orc_kp_generation(float *X, float *F, int32_t *rank, int N, int d, int m, const int32_t *p,
                      const int32_t *w, const int32_t *cap, const int32_t *order, const double *Z,
                      int nz, uint64_t seed, uint32_t gen, float p_c, float p_m)
{
    int n2 = 2 * N;
    float *RX = (float *)malloc((size_t)n2 * d * sizeof(float));
    float *RF = (float *)malloc((size_t)n2 * m * sizeof(float));
    int32_t *rr = (int32_t *)malloc((size_t)n2 * sizeof(int32_t));
    int32_t *sel = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    if (!RX || !RF || !rr || !sel) return ORC_ENOMEM;
    memcpy(RX, X, (size_t)N * d * sizeof(float));
    memcpy(RF, F, (size_t)N * m * sizeof(float));
    orc_kp_vary(X, rank, N, d, seed, gen, p_c, p_m, RX + (size_t)N * d);
    orc_kp_eval(RX + (size_t)N * d, N, d, m, p, w, cap, order, RF + (size_t)N * m);
    int rc = orc_select(RF, N, m, Z, nz, seed, gen, 0, 0, rr, sel, NULL, NULL, NULL);
    if (rc == ORC_OK) {
        for (int k = 0; k < N; ++k) {
            memcpy(X + (size_t)k * d, RX + (size_t)sel[k] * d, (size_t)d * sizeof(float));
            memcpy(F + (size_t)k * m, RF + (size_t)sel[k] * m, (size_t)m * sizeof(float));
            rank[k] = rr[sel[k]];
        }
    }
    free(RX); free(RF); free(rr); free(sel);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Hypervolume (minimisation) of the points P[n][m] inside the box below  */
/* ref, exact for m <= 3: m = 2 by a sweep over ascending f_0; m = 3 by    */
/* slices along f_2, each slice's area by the m = 2 sweep.  Returns -1   */
/* for m > 3.  App. E normalises it by prod_j (ref_j - ideal_j).          */
/* ---------------------------------------------------------------------- */
static int orc_cmp_f0(const void *a, const void *b)
{
    const double *x = (const double *)a, *y = (const double *)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    return (x[1] < y[1]) ? -1 : (x[1] > y[1]);
}

static double orc_hv2(double *pts, int n, const double *ref)
{
    qsort(pts, (size_t)n, 2 * sizeof(double), orc_cmp_f0);
    double area = 0.0, best = ref[1];
    for (int i = 0; i < n; ++i) {
        double x = pts[2 * i], y = pts[2 * i + 1];
        if (x >= ref[0] || y >= best) continue;
        area += (ref[0] - x) * (best - y);
        best = y;
    }
    return area;
}

double orc_hv(const float *P, int n, int m, const double *ref)
{
    if (m < 2 || m > 3 || n < 0) return -1.0;
    double *pts = (double *)malloc((size_t)(n > 0 ? n : 1) * 2 * sizeof(double));
    if (!pts) return -1.0;
    double hv = 0.0;
    if (m == 2) {
        for (int i = 0; i < n; ++i) {
            pts[2 * i] = P[(size_t)i * m];
            pts[2 * i + 1] = P[(size_t)i * m + 1];
        }
        hv = orc_hv2(pts, n, ref);
    } else {
        /* distinct f_2 levels below ref_2, ascending */
        double *lev = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
        if (!lev) { free(pts); return -1.0; }
        int nl = 0;
        for (int i = 0; i < n; ++i)
            if ((double)P[(size_t)i * m + 2] < ref[2]) lev[nl++] = P[(size_t)i * m + 2];
        for (int i = 1; i < nl; ++i) {  /* insertion sort */
            double x = lev[i];
            int k = i - 1;
            while (k >= 0 && lev[k] > x) { lev[k + 1] = lev[k]; --k; }
            lev[k + 1] = x;
        }
        for (int t = 0; t < nl; ++t) {
            if (t > 0 && lev[t] == lev[t - 1]) continue;
            int k = 0;
            for (int i = 0; i < n; ++i)
                if ((double)P[(size_t)i * m + 2] <= lev[t]) {
                    pts[2 * k] = P[(size_t)i * m];
                    pts[2 * k + 1] = P[(size_t)i * m + 1];
                    ++k;
                }
            double top = ref[2];
            for (int u = t + 1; u < nl; ++u)
                if (lev[u] > lev[t]) { top = lev[u]; break; }
            hv += orc_hv2(pts, k, ref) * (top - lev[t]);
        }
        free(lev);
    }
    free(pts);
    return hv;
}

/* ---------------------------------------------------------------------- */
/* IGD: mean over reference-front points of the Euclidean distance to the */
/* nearest population point (FP64).                                        */
/* ---------------------------------------------------------------------- */
double orc_igd(const float *P, int np, int m, const double *R, int nr)
{
    double acc = 0.0;
    for (int r = 0; r < nr; ++r) {
        double best = INFINITY;
        for (int i = 0; i < np; ++i) {
            double s = 0.0;
            for (int q = 0; q < m; ++q) {
                double t = (double)P[(size_t)i * m + q] - R[(size_t)r * m + q];
                double sq = t * t;
                s = s + sq;
            }
            if (s < best) best = s;
        }
        acc = acc + sqrt(best);
    }
    return nr > 0 ? acc / (double)nr : 0.0;
}
