/*
 * pa_oracle.c -- plain CPU oracle of population annealing (PA).
 * TEST INFRASTRUCTURE ONLY (see pa_oracle.h): tests, smoke() and the
 * cpu_baseline leg of bench.py call it; the product path never does.
 *
 * Every floating-point step is IEEE double with contraction disabled at build
 * time (-ffp-contract=off), so each expression below is rounded exactly as it
 * is written.
 */
#include "pa_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon et al., SC'11, "Parallel random numbers: as easy as
 * 1, 2, 3").  State (x0,x1,x2,x3), key (k0,k1).  One round multiplies x0 and
 * x2 by two fixed odd constants, keeps the four 32-bit halves, mixes the high
 * halves with the other words and the key, and advances the key by the two
 * Weyl constants.  Ten rounds.
 * ---------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t tag,
                 int32_t instance, uint32_t out[4])
{
    uint32_t ctr[4] = { c0, c1, c2, (tag << 28) | (uint32_t)instance };
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    or_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------
 * Schedule and tables.
 * beta_i = beta0 + (beta_max - beta0) * i / K  (Sec. 3: constant step).
 * Metropolis threshold T(beta, dE) = floor(exp(-beta dE) * 2^32), so that a
 * uniform 32-bit u accepts with probability exp(-beta dE) when u < T.
 * Weight D[j] = exp(-|dbeta| * 4 j): the factor exp[-(beta_i - beta_{i-1}) E]
 * of Eq. 3 relative to the reference energy, j = |k - kref| levels away
 * (energies are 4 apart): the lowest occupied level when cooling (dbeta >= 0),
 * the highest when heating (dbeta < 0), so the exponent is never positive.
 * ---------------------------------------------------------------------- */
double or_beta(const or_config* c, int32_t i)
{
    return c->beta0 + ((c->beta_max - c->beta0) * (double)i) / (double)c->K;
}

uint64_t or_threshold(double beta, int32_t dE)
{
    double x = -(beta * (double)dE);
    double t = floor(exp(x) * 4294967296.0);
    return (uint64_t)t;
}

double or_weight(double dbeta, int64_t j)
{
    return exp(-(fabs(dbeta) * (double)(4 * j)));
}

/* Number of energy levels: U (unsatisfied bonds) runs over 0..dim*N in steps
 * of two, so k = U >> 1 runs over 0..dim*N/2. */
int64_t or_num_bins(int32_t dim, int32_t L)
{
    int64_t N = 1;
    for (int d = 0; d < dim; ++d) N *= L;
    return (int64_t)dim * N / 2 + 1;
}

/* ------------------------------------------------------------------------
 * Lattice (Eq. 6).  Site s = x + L y (+ L^2 z); bond (s, d) joins s and
 * s + e_d (mod L) with coupling J[s*dim + d].  H = -sum_{s,d} J sigma sigma',
 * which is the -(J/2) sum' of Eq. 6 with its double count removed.
 * ---------------------------------------------------------------------- */
static int64_t site_count(int32_t dim, int32_t L)
{
    int64_t N = 1;
    for (int d = 0; d < dim; ++d) N *= L;
    return N;
}

static int64_t coord(int32_t L, int64_t s, int d)
{
    for (int k = 0; k < d; ++k) s /= L;
    return s % L;
}

static int64_t neighbour(int32_t L, int64_t s, int d, int dir)
{
    int64_t stride = 1;
    for (int k = 0; k < d; ++k) stride *= L;
    int64_t x = coord(L, s, d);
    int64_t xn = (x + dir + L) % L;
    return s + (xn - x) * stride;
}

static int colour_of(int32_t dim, int32_t L, int64_t s)
{
    int64_t sum = 0;
    for (int d = 0; d < dim; ++d) sum += coord(L, s, d);
    return (int)(sum & 1);
}

/* Neighbour table nb[(s*dim + d)*2 + 0/1] = s + e_d / s - e_d and the colour
 * of every site, built from neighbour()/colour_of() and kept for the last
 * (dim, L) asked for (the oracle is single-threaded). */
static struct { int32_t dim, L; int64_t* nb; int8_t* col; } geo = { 0, 0, NULL, NULL };

static void geometry(int32_t dim, int32_t L)
{
    if (geo.nb && geo.dim == dim && geo.L == L) return;
    free(geo.nb); free(geo.col);
    int64_t N = site_count(dim, L);
    geo.nb = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N * dim * 2));
    geo.col = (int8_t*)malloc((size_t)N);
    for (int64_t s = 0; s < N; ++s) {
        geo.col[s] = (int8_t)colour_of(dim, L, s);
        for (int d = 0; d < dim; ++d) {
            geo.nb[(s * dim + d) * 2 + 0] = neighbour(L, s, d, +1);
            geo.nb[(s * dim + d) * 2 + 1] = neighbour(L, s, d, -1);
        }
    }
    geo.dim = dim; geo.L = L;
}

void or_init_couplings(const or_config* c, int8_t* J)
{
    int64_t N = site_count(c->dim, c->L);
    for (int64_t s = 0; s < N; ++s)
        for (int d = 0; d < c->dim; ++d) {
            int8_t j = 1;
            if (c->model == OR_MODEL_PMJ) {
                uint32_t out[4];
                draw(c->coupling_seed, (uint32_t)(s >> 2), (uint32_t)d, 0u,
                     OR_TAG_COUPLING, c->instance_id, out);
                j = (out[s & 3] >> 31) ? -1 : 1;
            }
            J[s * c->dim + d] = j;
        }
}

/* Initial state at beta0 = 0: every state equally likely (Sec. 2), one
 * independent uniform bit per site.  The top bit of the draw set => -1.
 * Heating from near T = 0 starts from the ground state instead. */
void or_init_replica(const or_config* c, int64_t slot, int8_t* spins)
{
    int64_t N = site_count(c->dim, c->L);
    if (c->init == OR_INIT_GROUND) {
        for (int64_t s = 0; s < N; ++s) spins[s] = 1;
        return;
    }
    for (int64_t s = 0; s < N; ++s) {
        uint32_t out[4];
        draw(c->seed, (uint32_t)(s >> 2), 0u, (uint32_t)slot, OR_TAG_INIT,
             c->instance_id, out);
        spins[s] = (out[s & 3] >> 31) ? -1 : 1;
    }
}

void or_energy(int32_t dim, int32_t L, const int8_t* J, const int8_t* spins,
               int64_t* U, int64_t* M)
{
    int64_t N = site_count(dim, L);
    int64_t u = 0, m = 0;
    geometry(dim, L);
    for (int64_t s = 0; s < N; ++s) {
        m += spins[s];
        for (int d = 0; d < dim; ++d) {
            int64_t t = geo.nb[(s * dim + d) * 2 + 0];
            if (J[s * dim + d] * spins[s] * spins[t] < 0) ++u;
        }
    }
    *U = u;
    *M = m;
}

/* Energy change of flipping site s: 2 sigma_s sum_j J_sj sigma_j. */
int64_t or_delta_e(int32_t dim, int32_t L, const int8_t* J, const int8_t* spins, int64_t s)
{
    int64_t local = 0;
    geometry(dim, L);
    for (int d = 0; d < dim; ++d) {
        int64_t up = geo.nb[(s * dim + d) * 2 + 0];
        int64_t dn = geo.nb[(s * dim + d) * 2 + 1];
        local += J[s * dim + d] * spins[up];
        local += J[dn * dim + d] * spins[dn];
    }
    return 2 * spins[s] * local;
}

/* ------------------------------------------------------------------------
 * Metropolis equilibration (Sec. 2, theta sweeps at the new temperature).
 * One sweep = colour 0 sites (even coordinate sum) in ascending s, then
 * colour 1.  The random number of colour site s is word (h & 3) of the Philox
 * block with counter (2g + colour, h >> 2, SWEEP|id, slot), h = s >> 1, where
 * g is the global index of the sweep in the run.  It is drawn only when
 * dE > 0.
 * ---------------------------------------------------------------------- */
int64_t or_sweep_replica(const or_config* c, const int8_t* J, int8_t* spins,
                         int64_t slot, int64_t g0, int32_t nsweeps, const uint64_t T[3])
{
    int64_t N = site_count(c->dim, c->L);
    int64_t dU = 0;
    for (int32_t t = 0; t < nsweeps; ++t) {
        int64_t g = g0 + t;
        for (int colour = 0; colour < 2; ++colour) {
            int64_t cached = -1;
            uint32_t out[4] = { 0, 0, 0, 0 };
            for (int64_t s = 0; s < N; ++s) {
                geometry(c->dim, c->L);
                if (geo.col[s] != colour) continue;
                int64_t dE = or_delta_e(c->dim, c->L, J, spins, s);
                int accept;
                if (dE <= 0) {
                    accept = 1;
                } else {
                    int64_t h = s >> 1;
                    if ((h >> 2) != cached) {
                        cached = h >> 2;
                        const uint32_t ctr[4] = {
                            (uint32_t)(2 * g + colour), (uint32_t)(h >> 2),
                            (OR_TAG_SWEEP << 28) | (uint32_t)c->instance_id, (uint32_t)slot };
                        const uint32_t key[2] = { (uint32_t)(c->seed & 0xffffffffu),
                                                  (uint32_t)(c->seed >> 32) };
                        or_philox4x32_10(ctr, key, out);
                    }
                    uint64_t u = out[h & 3];
                    accept = u < T[dE / 4 - 1];
                }
                if (accept) {
                    spins[s] = (int8_t)-spins[s];
                    dU += dE / 2;
                }
            }
        }
    }
    return dU;
}

/* ------------------------------------------------------------------------
 * Eq. 3 / Eq. 4 on the energy histogram H (levels 4 apart).
 *   kref = lowest occupied level when cooling, highest when heating; every
 *   level on the far side of kref is empty.
 *   S = sum_k H_k D[|k - kref|]  (fixed order: 256 contiguous chunks of
 *   ceil(bins/256) levels, each summed left to right from 0.0, then the 256
 *   partial sums combined pairwise, level by level).
 *   tau_k = R0 D[|k - kref|] / S: Eq. 4 renormalised to the initial
 *   population R0, so that the expected population stays at R0 (Sec. 2 asks
 *   to keep it close to the original one).
 *   n_k = floor(tau_k), F_k = floor(frac(tau_k) * 2^32).
 * ---------------------------------------------------------------------- */
double or_tau_table(const uint32_t* H, int64_t bins, const double* Dtab, int64_t R0,
                    int32_t heating, uint32_t* n, uint32_t* F, int64_t* kref_out)
{
    int64_t kref = -1;
    if (heating) {
        for (int64_t k = bins - 1; k >= 0; --k)
            if (H[k] > 0) { kref = k; break; }
    } else {
        for (int64_t k = 0; k < bins; ++k)
            if (H[k] > 0) { kref = k; break; }
    }
    *kref_out = kref;
    if (kref < 0) {
        for (int64_t k = 0; k < bins; ++k) n[k] = F[k] = 0;
        return 0.0;
    }
    double part[256];
    int64_t ch = (bins + 255) / 256;
    for (int64_t ci = 0; ci < 256; ++ci) {
        double acc = 0.0;
        for (int64_t k = ci * ch; k < (ci + 1) * ch && k < bins; ++k) {
            int64_t j = heating ? kref - k : k - kref;
            if (j >= 0) acc = acc + (double)H[k] * Dtab[j];
        }
        part[ci] = acc;
    }
    for (int w = 256; w > 1; w /= 2)
        for (int j = 0; j < w / 2; ++j) part[j] = part[2 * j] + part[2 * j + 1];
    double S = part[0];
    for (int64_t k = 0; k < bins; ++k) {
        int64_t j = heating ? kref - k : k - kref;
        if (j < 0) { n[k] = F[k] = 0; continue; }
        double tau = ((double)R0 * Dtab[j]) / S;
        double nk = floor(tau);
        n[k] = (uint32_t)nk;
        F[k] = (uint32_t)floor((tau - nk) * 4294967296.0);
    }
    return S;
}

/* ------------------------------------------------------------------------
 * Adaptive temperature step (Sec. 3 points to the adaptive step of its
 * reference): keep the energy histograms of successive temperatures
 * overlapping by a target fraction.
 * ---------------------------------------------------------------------- */
double or_overlap(const uint32_t* H, int64_t bins, int64_t R, double dbeta)
{
    int heating = dbeta < 0.0;
    int64_t kref = -1;
    if (heating) {
        for (int64_t k = bins - 1; k >= 0; --k)
            if (H[k] > 0) { kref = k; break; }
    } else {
        for (int64_t k = 0; k < bins; ++k)
            if (H[k] > 0) { kref = k; break; }
    }
    if (kref < 0 || R < 1) return 0.0;
    double sw = 0.0;
    for (int64_t k = 0; k < bins; ++k) {
        int64_t j = heating ? kref - k : k - kref;
        if (j >= 0 && H[k]) sw = sw + (double)H[k] * or_weight(dbeta, j);
    }
    double a = 0.0;
    for (int64_t k = 0; k < bins; ++k) {
        int64_t j = heating ? kref - k : k - kref;
        if (j < 0 || !H[k]) continue;
        double p = (double)H[k] / (double)R;
        double q = ((double)H[k] * or_weight(dbeta, j)) / sw;
        a = a + (p < q ? p : q);
    }
    return a;
}

double or_adaptive_next(const uint32_t* H, int64_t bins, int64_t R, double beta,
                        double beta_end, double target)
{
    double span = beta_end - beta;
    if (span == 0.0) return beta;
    if (or_overlap(H, bins, R, span) >= target) return beta_end;
    double lo = 0.0, hi = fabs(span), sgn = span < 0.0 ? -1.0 : 1.0;
    for (int it = 0; it < 60; ++it) {
        double mid = lo + (hi - lo) * 0.5;
        if (or_overlap(H, bins, R, sgn * mid) >= target) lo = mid;
        else hi = mid;
    }
    return beta + sgn * lo;
}

/* Nearest-integer resampling (the Poisson draw of Sec. 2 replaced by one of
 * its variants): r_i = n_k + [u_i < F_k], u_i = word (i & 3) of the Philox
 * block (i >> 2, step, 0, RESAMPLE|id).  E[r_i] = tau_k. */
void or_copy_counts(const or_config* c, int32_t step, const uint32_t* ebin, int64_t R,
                    const uint32_t* n, const uint32_t* F, uint32_t* r)
{
    for (int64_t i = 0; i < R; ++i) {
        uint32_t out[4];
        draw(c->seed, (uint32_t)(i >> 2), (uint32_t)step, 0u, OR_TAG_RESAMPLE,
             c->instance_id, out);
        uint32_t u = out[i & 3];
        uint32_t k = ebin[i];
        r[i] = n[k] + (u < F[k] ? 1u : 0u);
    }
}

/* Poisson(1) distribution function, term by term: P(X <= m) = sum_{j<=m}
 * e^-1 / j!, each term the previous one divided by j, the sum in the order
 * of m.  Entries are scaled to 32-bit thresholds and truncated. */
int32_t or_poisson1_thresholds(uint32_t* T, int32_t cap)
{
    double term = exp(-1.0), cdf = 0.0;
    for (int32_t m = 0; m < cap; ++m) {
        if (m > 0) term = term / (double)m;
        cdf = cdf + term;
        double scaled = floor(ldexp(cdf, 32));
        T[m] = scaled >= 4294967295.0 ? 0xffffffffu : (uint32_t)scaled;
        if (T[m] == 0xffffffffu) return m + 1;
    }
    return cap;
}

/* Poisson resampling, the draw Sec. 2 prescribes: r_i ~ Poisson(tau_k) with
 * tau_k = n_k + f_k, f_k = F_k / 2^32.  A Poisson(tau) count is the number of
 * events of a unit-rate Poisson process on [0, tau]: every unit interval adds
 * an independent Poisson(1) count, drawn by inversion (the smallest m with
 * u < T[m]), and the last interval of length f_k adds a Poisson(f_k) count,
 * drawn as a Poisson(1) count whose events are kept with probability f_k
 * (thinning: keep when u < F_k).  The uniforms u_0, u_1, ... of replica i are
 * the words of the Philox blocks (i, step, b, POISSON|id), b = 0, 1, ...,
 * taken in order: first the fractional interval's count, then its thinning
 * draws, then the n_k unit-interval counts. */
typedef struct {
    const or_config* c;
    uint32_t i, step, b, w;
    uint32_t out[4];
} or_ustream;

static uint32_t next_u(or_ustream* s)
{
    if (s->w == 4) {
        draw(s->c->seed, s->i, s->step, s->b, OR_TAG_POISSON, s->c->instance_id, s->out);
        s->b++;
        s->w = 0;
    }
    return s->out[s->w++];
}

static uint32_t poisson1(or_ustream* s, const uint32_t* T, int32_t len)
{
    uint32_t u = next_u(s);
    uint32_t m = 0;
    while ((int32_t)m < len && u >= T[m]) ++m;
    return m;
}

void or_copy_counts_poisson(const or_config* c, int32_t step, const uint32_t* ebin, int64_t R,
                            const uint32_t* n, const uint32_t* F, uint32_t* r)
{
    uint32_t T[64];
    int32_t len = or_poisson1_thresholds(T, 64);
    for (int64_t i = 0; i < R; ++i) {
        or_ustream s = { c, (uint32_t)i, (uint32_t)step, 0u, 4u, { 0, 0, 0, 0 } };
        uint32_t k = ebin[i];
        uint32_t count = 0;
        uint32_t events = poisson1(&s, T, len);          /* interval of length 1 ... */
        for (uint32_t e = 0; e < events; ++e)           /* ... thinned to f_k       */
            if (next_u(&s) < F[k]) ++count;
        for (uint32_t j = 0; j < n[k]; ++j) count += poisson1(&s, T, len);
        r[i] = count;
    }
}

/* Multinomial resampling, a variant of the Poisson draw (Sec. 2 refers to
 * the review of Machta for these modifications): the new population is R0
 * independent draws from the old one, replica i drawn with probability
 * tau_i / sum_j tau_j, so its size is exactly R0.  tau_i enters in 32.32
 * fixed point, t_i = n_k 2^32 + F_k for the level k of replica i, which makes
 * the cumulative weights C_i = t_0 + ... + t_i exact integers.  Draw j
 * (j = 0 .. R0 - 1) takes the 64-bit uniform v = w[2(j & 1)] + 2^32
 * w[2(j & 1) + 1] of the Philox block (j >> 1, step, 0, MULTINOMIAL|id), the
 * point x = floor(v C_{R-1} / 2^64) in [0, C_{R-1}), and gives one copy to the
 * first replica i with C_i > x. */
void or_copy_counts_multinomial(const or_config* c, int32_t step, const uint32_t* ebin, int64_t R,
                                const uint32_t* n, const uint32_t* F, uint32_t* r)
{
    uint64_t* C = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(R > 0 ? R : 1));
    uint64_t total = 0;
    for (int64_t i = 0; i < R; ++i) {
        uint32_t k = ebin[i];
        total += ((uint64_t)n[k] << 32) + (uint64_t)F[k];
        C[i] = total;
        r[i] = 0;
    }
    if (R < 1 || total == 0) { free(C); return; }
    for (int64_t j = 0; j < c->R0; ++j) {
        uint32_t out[4];
        draw(c->seed, (uint32_t)(j >> 1), (uint32_t)step, 0u, OR_TAG_MULTINOMIAL, c->instance_id,
             out);
        uint64_t v = (uint64_t)out[2 * (j & 1)] | ((uint64_t)out[2 * (j & 1) + 1] << 32);
        uint64_t x = (uint64_t)(((unsigned __int128)v * (unsigned __int128)total) >> 64);
        int64_t lo = 0, hi = R - 1;          /* first i with C[i] > x */
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (C[mid] > x) hi = mid;
            else lo = mid + 1;
        }
        r[lo] += 1;
    }
    free(C);
}

/* Population averages (Sec. 2) from exact integer sums. */
void or_derive_obs(or_obs* o, int64_t N)
{
    double Rd = (double)o->R, Nd = (double)N;
    double mE = (double)o->sumE / Rd;
    double mE2 = (double)o->sumE2 / Rd;
    double mA = (double)o->sumAbsM / Rd;
    double mM2 = (double)o->sumM2 / Rd;
    o->e = mE / Nd;
    o->cv = ((o->beta * o->beta) * (mE2 - mE * mE)) / Nd;
    o->m_abs = mA / Nd;
    o->chi = (o->beta * (mM2 - mA * mA)) / Nd;
}

/* ------------------------------------------------------------------------
 * A whole run.
 * ---------------------------------------------------------------------- */
struct or_run {
    or_config c;
    int64_t N, bins, cap, R, R_prev, g, kref, parity, fails;
    int32_t step;
    int8_t *J, *spins, *spins2;
    uint32_t *ebin, *ebin2, *H, *r, *o, *tn, *tF;
    int32_t *M, *M2;
    int64_t *U, *U2;       /* energies tracked through the sweeps */
    uint64_t *T;           /* [(K+1) * 3] */
    double *betas;         /* [K+1] inverse temperature of every step */
    double S, lnQ, lnZ;
    or_obs obs;
};

static void measure(or_run* r)
{
    memset(r->H, 0, sizeof(uint32_t) * (size_t)r->bins);
    or_obs* o = &r->obs;
    o->step = r->step;
    o->R = r->R;
    o->sumE = o->sumE2 = o->sumAbsM = o->sumM2 = 0;
    for (int64_t i = 0; i < r->R; ++i) {
        int64_t U, M;
        or_energy(r->c.dim, r->c.L, r->J, r->spins + i * r->N, &U, &M);
        if (U != r->U[i]) ++r->fails;            /* from scratch == tracked */
        if ((U & 1) != r->parity) ++r->fails;    /* parity is a constant   */
        r->U[i] = U;
        r->ebin[i] = (uint32_t)(U >> 1);
        r->M[i] = (int32_t)M;
        r->H[U >> 1] += 1;
        int64_t E = 2 * U - (int64_t)r->c.dim * r->N;
        o->sumE += E;
        o->sumE2 += E * E;
        o->sumAbsM += M < 0 ? -M : M;
        o->sumM2 += M * M;
    }
    o->beta = r->betas[r->step];
    o->lnQ = r->lnQ;
    o->lnZ = r->lnZ;
    or_derive_obs(o, r->N);
}

or_run* or_create(const or_config* c)
{
    if (c->dim != 2 && c->dim != 3) return NULL;
    if (c->L < 2 || (c->L & 1)) return NULL;
    if (c->K < 1 || c->theta < 0 || c->R0 < 1) return NULL;
    if (c->instance_id < 0 || c->instance_id >= (1 << 28)) return NULL;
    if (c->init != OR_INIT_RANDOM && c->init != OR_INIT_GROUND) return NULL;
    if (c->init == OR_INIT_GROUND && c->model != OR_MODEL_FERRO) return NULL;
    if (c->resample != OR_RESAMPLE_NEAREST && c->resample != OR_RESAMPLE_POISSON &&
        c->resample != OR_RESAMPLE_MULTINOMIAL)
        return NULL;
    or_run* r = (or_run*)calloc(1, sizeof(or_run));
    r->c = *c;
    r->N = site_count(c->dim, c->L);
    r->bins = or_num_bins(c->dim, c->L);
    r->cap = c->capacity > 0 ? c->capacity
                             : c->R0 + 16 * (int64_t)ceil(sqrt((double)c->R0)) + 1024;
    if (r->cap < c->R0) { free(r); return NULL; }
    size_t cap = (size_t)r->cap, N = (size_t)r->N, bins = (size_t)r->bins;
    r->J = (int8_t*)malloc(N * (size_t)c->dim);
    r->spins = (int8_t*)malloc(cap * N);
    r->spins2 = (int8_t*)malloc(cap * N);
    r->ebin = (uint32_t*)calloc(cap, 4);
    r->ebin2 = (uint32_t*)calloc(cap, 4);
    r->M = (int32_t*)calloc(cap, 4);
    r->M2 = (int32_t*)calloc(cap, 4);
    r->U = (int64_t*)calloc(cap, 8);
    r->U2 = (int64_t*)calloc(cap, 8);
    r->r = (uint32_t*)calloc(cap, 4);
    r->o = (uint32_t*)calloc(cap, 4);
    r->H = (uint32_t*)calloc(bins, 4);
    r->tn = (uint32_t*)calloc(bins, 4);
    r->tF = (uint32_t*)calloc(bins, 4);
    r->T = (uint64_t*)calloc((size_t)(c->K + 1) * 3, 8);
    r->betas = (double*)calloc((size_t)(c->K + 1), 8);
    for (int32_t i = 0; i <= c->K; ++i) {
        r->betas[i] = or_beta(c, i);
        for (int cl = 0; cl < 3; ++cl)
            r->T[i * 3 + cl] = or_threshold(r->betas[i], 4 * (cl + 1));
    }
    or_init_couplings(c, r->J);
    r->R = c->R0;
    r->kref = -1;
    for (int64_t i = 0; i < r->R; ++i) or_init_replica(c, i, r->spins + i * r->N);
    /* the parity of U is fixed by the couplings: read it off replica 0 */
    {
        int64_t U, M;
        or_energy(c->dim, c->L, r->J, r->spins, &U, &M);
        r->parity = U & 1;
    }
    for (int64_t i = 0; i < r->R; ++i) {
        int64_t U, M;
        or_energy(c->dim, c->L, r->J, r->spins + i * r->N, &U, &M);
        r->U[i] = U;
    }
    r->lnQ = 0.0;
    /* ln Z at beta0: N ln 2 states at infinite temperature; near T = 0 the two
     * ground states (all up, all down) of energy -dim N (Sec. 2, Eq. 5's
     * initial value ln Omega of each protocol). */
    if (c->init == OR_INIT_GROUND)
        r->lnZ = log(2.0) + c->beta0 * (double)((int64_t)c->dim * r->N);
    else
        r->lnZ = (double)r->N * log(2.0);
    measure(r);
    return r;
}

void or_destroy(or_run* r)
{
    if (!r) return;
    free(r->J); free(r->spins); free(r->spins2); free(r->ebin); free(r->ebin2);
    free(r->M); free(r->M2); free(r->U); free(r->U2); free(r->r); free(r->o);
    free(r->H); free(r->tn); free(r->tF); free(r->T); free(r->betas);
    free(r);
}

int or_resample_to(or_run* r, double beta_next)
{
    int32_t i = r->step + 1;
    if (i > r->c.K) return -2;
    r->betas[i] = beta_next;
    for (int cl = 0; cl < 3; ++cl) r->T[i * 3 + cl] = or_threshold(beta_next, 4 * (cl + 1));
    return or_resample(r);
}

double or_current_beta(const or_run* r) { return r->betas[r->step]; }

int or_resample(or_run* r)
{
    const or_config* c = &r->c;
    int32_t i = r->step + 1;
    if (i > c->K) return -2;
    if (r->R < 1) return -4;
    double dbeta = r->betas[i] - r->betas[i - 1];
    double* Dtab = (double*)malloc(sizeof(double) * (size_t)r->bins);
    for (int64_t j = 0; j < r->bins; ++j) Dtab[j] = or_weight(dbeta, j);
    int64_t hsum = 0;
    for (int64_t k = 0; k < r->bins; ++k) hsum += r->H[k];
    if (hsum != r->R) ++r->fails;                /* sum_k H_k = R */
    r->S = or_tau_table(r->H, r->bins, Dtab, c->R0, dbeta < 0.0, r->tn, r->tF, &r->kref);
    free(Dtab);
    int64_t Eref = 2 * (2 * r->kref + r->parity) - (int64_t)c->dim * r->N;
    r->lnQ = (log(r->S) - log((double)r->R)) - dbeta * (double)Eref;   /* Eq. 3 */
    r->lnZ = r->lnZ + r->lnQ;                                          /* Eq. 5 */
    if (c->resample == OR_RESAMPLE_POISSON)
        or_copy_counts_poisson(c, i, r->ebin, r->R, r->tn, r->tF, r->r);
    else if (c->resample == OR_RESAMPLE_MULTINOMIAL)
        or_copy_counts_multinomial(c, i, r->ebin, r->R, r->tn, r->tF, r->r);
    else
        or_copy_counts(c, i, r->ebin, r->R, r->tn, r->tF, r->r);
    int64_t total = 0;
    for (int64_t j = 0; j < r->R; ++j) {
        r->o[j] = (uint32_t)total;
        total += r->r[j];
    }
    r->R_prev = r->R;
    r->step = i;
    if (total > r->cap) return -3;
    /* exact copies (Sec. 2): copy j of replica i lands in slot o_i + j */
    for (int64_t j = 0; j < r->R; ++j)
        for (uint32_t k = 0; k < r->r[j]; ++k) {
            int64_t dst = (int64_t)r->o[j] + k;
            memcpy(r->spins2 + dst * r->N, r->spins + j * r->N, (size_t)r->N);
            r->ebin2[dst] = r->ebin[j];
            r->M2[dst] = r->M[j];
            r->U2[dst] = r->U[j];
        }
    int8_t* ts = r->spins; r->spins = r->spins2; r->spins2 = ts;
    uint32_t* te = r->ebin; r->ebin = r->ebin2; r->ebin2 = te;
    int32_t* tm = r->M; r->M = r->M2; r->M2 = tm;
    int64_t* tu = r->U; r->U = r->U2; r->U2 = tu;
    r->R = total;
    if (total < 1) return -4;
    return 0;
}

/* Replica exchange between GPUs (Sec. 3), on a population whose N "GPUs" are
 * consecutive slot ranges: after a resample the replicas are put in a new slot
 * order, given as segments of the current order -- new slots are filled in
 * order with old slots src[q] .. src[q] + len[q] - 1, q = 0 .. nseg - 1.  The
 * population's states, levels, magnetisations and tracked energies move with
 * the slots.  Returns 0, or -1 if a segment leaves [0, R) or the lengths do not
 * add up to R. */
int or_permute(or_run* r, int32_t nseg, const int64_t* src, const int64_t* len)
{
    int64_t total = 0;
    for (int32_t q = 0; q < nseg; ++q) {
        if (len[q] < 0 || src[q] < 0 || src[q] + len[q] > r->R) return -1;
        total += len[q];
    }
    if (total != r->R) return -1;
    int64_t dst = 0;
    for (int32_t q = 0; q < nseg; ++q)
        for (int64_t k = 0; k < len[q]; ++k, ++dst) {
            int64_t from = src[q] + k;
            memcpy(r->spins2 + dst * r->N, r->spins + from * r->N, (size_t)r->N);
            r->ebin2[dst] = r->ebin[from];
            r->M2[dst] = r->M[from];
            r->U2[dst] = r->U[from];
        }
    int8_t* ts = r->spins; r->spins = r->spins2; r->spins2 = ts;
    uint32_t* te = r->ebin; r->ebin = r->ebin2; r->ebin2 = te;
    int32_t* tm = r->M; r->M = r->M2; r->M2 = tm;
    int64_t* tu = r->U; r->U = r->U2; r->U2 = tu;
    return 0;
}

int or_sweep(or_run* r, int32_t nsweeps)
{
    if (nsweeps < 0) return -1;
    const uint64_t* T = r->T + (size_t)r->step * 3;
    for (int64_t i = 0; i < r->R; ++i)
        r->U[i] += or_sweep_replica(&r->c, r->J, r->spins + i * r->N, i, r->g, nsweeps, T);
    r->g += nsweeps;
    measure(r);
    return 0;
}

int or_step(or_run* r)
{
    int rc = or_resample(r);
    if (rc) return rc;
    return or_sweep(r, r->c.theta);
}

void or_observables(const or_run* r, or_obs* out) { *out = r->obs; }

int64_t or_R(const or_run* r) { return r->R; }
int64_t or_N(const or_run* r) { return r->N; }
int64_t or_bins(const or_run* r) { return r->bins; }
int32_t or_step_index(const or_run* r) { return r->step; }
int64_t or_sweep_counter(const or_run* r) { return r->g; }
const int8_t* or_spins(const or_run* r) { return r->spins; }
const uint32_t* or_ebin(const or_run* r) { return r->ebin; }
const int32_t* or_mag(const or_run* r) { return r->M; }
const uint32_t* or_hist(const or_run* r) { return r->H; }
const uint32_t* or_counts(const or_run* r) { return r->r; }
const uint32_t* or_offsets(const or_run* r) { return r->o; }
const uint32_t* or_tab_n(const or_run* r) { return r->tn; }
const uint32_t* or_tab_F(const or_run* r) { return r->tF; }
const int8_t* or_couplings(const or_run* r) { return r->J; }
int64_t or_R_prev(const or_run* r) { return r->R_prev; }
int64_t or_kref(const or_run* r) { return r->kref; }
double or_S(const or_run* r) { return r->S; }
int64_t or_parity(const or_run* r) { return r->parity; }
int64_t or_check_failures(const or_run* r) { return r->fails; }
double or_lnQ(const or_run* r) { return r->lnQ; }
double or_lnZ(const or_run* r) { return r->lnZ; }
