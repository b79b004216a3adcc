/*
 * FP64 CPU oracle for the lazy-PCA / Gibbs denoising sampler.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * restatement of what the sampler computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant generator with the CUDA library, and the
 * CUDA library never calls it.
 *
 * What it follows (arXiv 2507.14869):
 *   - Posterior Hamiltonian, Eq. (denoising_posterior_Hamiltonian): prior pair
 *     potential plus data term (g_i - x_i)^2 / (2 sigma^2).
 *   - Single-site Gibbs conditional, Eq. (gibbs_sampler_elementary_step):
 *     weight exp{ sum_{j~i} 2 beta J 1{s = x_j} - (g_i - s)^2/(2 sigma^2) }.
 *   - Lazy PCA transition, Eq. (posterior_pca_transition_matrix) and the
 *     Section 5.2 transition: every site independently draws from the same
 *     conditional evaluated on the previous configuration, with the inertial
 *     price beta*q*1{s != x_i} (the subscript printed as x_j is read as the
 *     site's own previous label x_i, as in Section 3 "The lazy PCA").
 *   - Potts pair potential Eq. (prior_pair_potential); 4- or 8-neighbourhood
 *     Eq. (neighborhood) with missing neighbours dropped at the edge.
 *   Extensions named by the workloads, not printed in the paper: the
 *   truncated-linear pair potential c_T min(|s-t|, T) (Section 7 lists L1-type
 *   priors as future work) and the binary-symmetric (flip) channel.
 *
 * Energies (lower = likelier), for site i, candidate label s:
 *   E_i(s) = prior_i(s) + data_i(s) + lambda * 1{s != x_i}
 *   prior_i(s) = -c_P * #{j in N(i): x_j = s}           (Potts, c_P = 2 beta J)
 *              =  c_T * sum_{j in N(i)} min(|s - x_j|, T) (truncated linear)
 *   data_i(s)  = a * (g_i - s)^2, a = 1 / (2 sigma^2)      (Gaussian, label units)
 *              = -ln(1-p) if s = g_i, else -ln p          (flip channel)
 * Draw: w_s = exp(-(E_s - E_min)), C_k = sum_{s<=k} w_s in label order,
 * Z = C_{L-1}, t = u Z, new label = smallest k with t < C_k.  The uniform u
 * is the top 24 bits of one Philox4x32-10 output word times 2^-24.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC 2011), written here from its published
 * definition.  Counter = (col >> 2, row, sweep, (tag << 24) | chain), key =
 * (seed low 32 bits, seed high 32 bits), word = col & 3; tag 0 = PCA,
 * 1 = Gibbs.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared [-fopenmp] -lm.  Contraction
 * must stay off so that every product and sum is rounded once, as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_POTTS 0
#define ORC_TRUNC_LINEAR 1
#define ORC_GAUSS 0
#define ORC_FLIP 1
#define ORC_NONE 2   /* no likelihood: the prior alone */
#define ORC_TAG_PCA 0u
#define ORC_TAG_GIBBS 1u
#define ORC_NEAR 1e-6

typedef struct {
    int L;            /* number of labels, 2..256 */
    int nbhd;         /* 4 or 8 */
    int pair;         /* ORC_POTTS or ORC_TRUNC_LINEAR */
    int pair_T;       /* truncation T (truncated linear) */
    int noise;        /* ORC_GAUSS, ORC_FLIP or ORC_NONE */
    int inertia_norm; /* 0: lambda 1{s != x_i}; p = 1, 2: lambda (|s - x_i| / (L-1))^p */
    double pair_coef; /* c_P (Potts reward) or c_T (slope) */
    double sigma;     /* Gaussian std, label units */
    double flip_p;    /* flip probability */
    double inertia;   /* lambda = beta q */
} orc_model;

/* ------------------------------------------------------------------ Philox */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {               /* Weyl key schedule */
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in [0,1) with 24 bits: exact in both FP32 and FP64. */
double orc_uniform(uint64_t seed, uint32_t chain, uint32_t tag, uint32_t sweep,
                   uint32_t row, uint32_t col)
{
    uint32_t ctr[4] = { col >> 2, row, sweep, (tag << 24) | (chain & 0xFFFFFFu) };
    uint32_t key[2] = { (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32) };
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    uint32_t word = out[col & 3u];
    return (double)(word >> 8) * (1.0 / 16777216.0);
}

/* ------------------------------------------------------ per-site conditional */

/* Energies E_i(s) for s = 0..L-1 (eq. gibbs_sampler_elementary_step with the
 * lazy-PCA inertial term of Section 5.2).  nb holds the labels of the nnb
 * neighbours that exist (free boundary).  lam is the inertia (0 for Gibbs):
 * the L0 price lam 1{s != x_i} of Section 3, or with inertia_norm p = 1, 2
 * the Lp price lam (|s - x_i| / (L - 1))^p on intensities (Section 3, the
 * norms proportional to the size of the change). */
static void site_energies(const orc_model *m, int g, int xi, const int *nb, int nnb,
                          double lam, double *E)
{
    const double a = 1.0 / (2.0 * m->sigma * m->sigma);
    const double u_same = -log(1.0 - m->flip_p);
    const double u_diff = -log(m->flip_p);
    for (int s = 0; s < m->L; ++s) {
        double prior;
        if (m->pair == ORC_POTTS) {
            int n = 0;
            for (int j = 0; j < nnb; ++j)
                n += (nb[j] == s);
            prior = -(m->pair_coef * (double)n);
        } else {
            int P = 0;
            for (int j = 0; j < nnb; ++j) {
                int d = abs(s - nb[j]);
                P += d < m->pair_T ? d : m->pair_T;
            }
            prior = m->pair_coef * (double)P;
        }
        double data;
        if (m->noise == ORC_GAUSS) {
            int dg = g - s;
            data = a * (double)(dg * dg);
        } else if (m->noise == ORC_FLIP) {
            data = (s == g) ? u_same : u_diff;
        } else {
            data = 0.0;
        }
        double inert;
        if (m->inertia_norm == 0) {
            inert = (s != xi) ? lam : 0.0;
        } else {
            const double d = (double)abs(s - xi) / (double)(m->L - 1);
            inert = lam * (m->inertia_norm == 1 ? d : d * d);
        }
        E[s] = (prior + data) + inert;
    }
}

/* Normalised conditional probabilities p(s) (for exact transition matrices). */
void orc_site_probs(const orc_model *m, int g, int xi, const int *nb, int nnb,
                    double lam, double *p)
{
    double E[256];
    site_energies(m, g, xi, nb, nnb, lam, E);
    double Emin = E[0];
    for (int s = 1; s < m->L; ++s)
        if (E[s] < Emin) Emin = E[s];
    double Z = 0.0;
    for (int s = 0; s < m->L; ++s) {
        p[s] = exp(-(E[s] - Emin));
        Z += p[s];
    }
    for (int s = 0; s < m->L; ++s)
        p[s] /= Z;
}

/* Inverse-CDF draw with uniform u.  *near is set when u lies within 1e-6 of
 * the normalised CDF boundary just above or just below the chosen label. */
int orc_site_draw(const orc_model *m, int g, int xi, const int *nb, int nnb,
                  double lam, double u, int *near)
{
    double E[256], C[256];
    site_energies(m, g, xi, nb, nnb, lam, E);
    double Emin = E[0];
    for (int s = 1; s < m->L; ++s)
        if (E[s] < Emin) Emin = E[s];
    double acc = 0.0;
    for (int s = 0; s < m->L; ++s) {
        acc += exp(-(E[s] - Emin));
        C[s] = acc;
    }
    const double Z = C[m->L - 1];
    const double t = u * Z;
    int k = 0;
    while (k < m->L - 1 && !(t < C[k]))
        ++k;
    if (near) {
        int nr = fabs(u - C[k] / Z) < ORC_NEAR;
        if (k > 0 && fabs(u - C[k - 1] / Z) < ORC_NEAR)
            nr = 1;
        *near = nr;
    }
    return k;
}

/* Labels of the neighbours of (r, c) that exist, in a fixed order. */
static int gather(const uint8_t *x, int H, int W, int nbhd, int r, int c, int *nb)
{
    static const int dr8[8] = { -1, 1, 0, 0, -1, -1, 1, 1 };
    static const int dc8[8] = { 0, 0, -1, 1, -1, 1, -1, 1 };
    int n = 0;
    for (int j = 0; j < nbhd; ++j) {
        int rr = r + dr8[j], cc = c + dc8[j];
        if (rr < 0 || rr >= H || cc < 0 || cc >= W)
            continue;
        nb[n++] = x[(size_t)rr * W + cc];
    }
    return n;
}

/* ------------------------------------------------------------------ sweeps */

/* One lazy-PCA sweep (eq. posterior_pca_transition_matrix): every site draws
 * from its conditional on x (the previous configuration) into xn.
 * near (nullable) receives the per-site near-boundary flags.
 * Returns the number of near-boundary draws. */
long orc_pca_sweep(const orc_model *m, int H, int W, const uint8_t *g,
                   const uint8_t *x, uint8_t *xn, uint64_t seed, uint32_t chain,
                   uint32_t sweep, uint8_t *near)
{
    long n_near = 0;
#pragma omp parallel for schedule(static) reduction(+:n_near) if ((long)H * W >= 16384)
    for (int r = 0; r < H; ++r) {
        int nb[8];
        for (int c = 0; c < W; ++c) {
            size_t i = (size_t)r * W + c;
            int nnb = gather(x, H, W, m->nbhd, r, c, nb);
            double u = orc_uniform(seed, chain, ORC_TAG_PCA, sweep, (uint32_t)r, (uint32_t)c);
            int nr = 0;
            xn[i] = (uint8_t)orc_site_draw(m, g[i], x[i], nb, nnb, m->inertia, u, &nr);
            if (near) near[i] = (uint8_t)nr;
            n_near += nr;
        }
    }
    return n_near;
}

/* Lazy-PCA draws for a list of sites only (sampled parity on large images). */
long orc_pca_sites(const orc_model *m, int H, int W, const uint8_t *g, const uint8_t *x,
                   long n_sites, const int32_t *rows, const int32_t *cols,
                   uint64_t seed, uint32_t chain, uint32_t sweep,
                   uint8_t *out, uint8_t *near)
{
    long n_near = 0;
#pragma omp parallel for schedule(static) reduction(+:n_near) if (n_sites >= 4096)
    for (long k = 0; k < n_sites; ++k) {
        int nb[8];
        int r = rows[k], c = cols[k];
        size_t i = (size_t)r * W + c;
        int nnb = gather(x, H, W, m->nbhd, r, c, nb);
        double u = orc_uniform(seed, chain, ORC_TAG_PCA, sweep, (uint32_t)r, (uint32_t)c);
        int nr = 0;
        out[k] = (uint8_t)orc_site_draw(m, g[i], x[i], nb, nnb, m->inertia, u, &nr);
        if (near) near[k] = (uint8_t)nr;
        n_near += nr;
    }
    return n_near;
}

/* Colour of a site for the colour-ordered Gibbs scan: 2 colours by (r+c)
 * parity for the 4-neighbourhood, 4 colours by (r mod 2, c mod 2) for the
 * 8-neighbourhood.  No two sites of one colour are neighbours. */
static int site_colour(int nbhd, int r, int c)
{
    return nbhd == 4 ? ((r + c) & 1) : (((r & 1) << 1) | (c & 1));
}

static long gibbs_visit(const orc_model *m, int H, int W, const uint8_t *g, uint8_t *x,
                        uint64_t seed, uint32_t chain, uint32_t sweep, int r, int c,
                        uint8_t *near)
{
    int nb[8];
    size_t i = (size_t)r * W + c;
    int nnb = gather(x, H, W, m->nbhd, r, c, nb);
    double u = orc_uniform(seed, chain, ORC_TAG_GIBBS, sweep, (uint32_t)r, (uint32_t)c);
    int nr = 0;
    x[i] = (uint8_t)orc_site_draw(m, g[i], x[i], nb, nnb, 0.0, u, &nr);
    if (near) near[i] = (uint8_t)nr;
    return nr;
}

/* One systematic single-site Gibbs sweep, in place (Section 5.1): every
 * site is visited once, in row-major order (order 0), column-major order
 * (order 1, the example order of Section 4) or colour order (order 2).
 * Returns the number of near-boundary draws. */
long orc_gibbs_sweep(const orc_model *m, int H, int W, const uint8_t *g, uint8_t *x,
                     uint64_t seed, uint32_t chain, uint32_t sweep, int order,
                     uint8_t *near)
{
    long n_near = 0;
    if (order == 0) {
        for (int r = 0; r < H; ++r)
            for (int c = 0; c < W; ++c)
                n_near += gibbs_visit(m, H, W, g, x, seed, chain, sweep, r, c, near);
    } else if (order == 1) {
        for (int c = 0; c < W; ++c)
            for (int r = 0; r < H; ++r)
                n_near += gibbs_visit(m, H, W, g, x, seed, chain, sweep, r, c, near);
    } else {
        int ncol = m->nbhd == 4 ? 2 : 4;
        for (int q = 0; q < ncol; ++q)
            for (int r = 0; r < H; ++r)
                for (int c = 0; c < W; ++c)
                    if (site_colour(m->nbhd, r, c) == q)
                        n_near += gibbs_visit(m, H, W, g, x, seed, chain, sweep, r, c, near);
    }
    return n_near;
}

/* Run a chain for nsweeps sweeps starting at sweep counter t0.  x holds the
 * state (in/out); acc accumulates x after every completed sweep whose
 * 1-based index exceeds burn_in (posterior-mean estimator, Section 2
 * "Bayesian inference").  sampler 0 = lazy PCA, 1 = Gibbs with gibbs_order.
 * Returns the number of near-boundary draws. */
long orc_run_chain(const orc_model *m, int H, int W, const uint8_t *g, uint8_t *x,
                   double *acc, uint64_t seed, uint32_t chain, uint32_t t0,
                   int nsweeps, int burn_in, int sampler, int gibbs_order)
{
    size_t n = (size_t)H * W;
    uint8_t *tmp = (uint8_t *)malloc(n ? n : 1);
    long n_near = 0;
    for (int k = 0; k < nsweeps; ++k) {
        uint32_t t = t0 + (uint32_t)k;
        if (sampler == 0) {
            n_near += orc_pca_sweep(m, H, W, g, x, tmp, seed, chain, t, NULL);
            memcpy(x, tmp, n);
        } else {
            n_near += orc_gibbs_sweep(m, H, W, g, x, seed, chain, t, gibbs_order, NULL);
        }
        if ((long)t + 1 > (long)burn_in && acc)
            for (size_t i = 0; i < n; ++i)
                acc[i] += (double)x[i];
    }
    free(tmp);
    return n_near;
}

/* Histogram of visited states of a tiny lattice (L^(H*W) <= 2^22 states):
 * state index = sum_i x_i L^i over sites i in row-major order.  Used to
 * compare the chain's empirical law with exact enumeration. */
long orc_state_histogram(const orc_model *m, int H, int W, const uint8_t *g, uint8_t *x,
                         uint64_t seed, uint32_t chain, int nsweeps, int sampler,
                         int gibbs_order, double *hist)
{
    size_t n = (size_t)H * W;
    uint8_t tmp[32];
    long n_near = 0;
    double nstates = pow((double)m->L, (double)n);
    if (n > 32 || nstates > 4194304.0)
        return -1;
    for (int k = 0; k < nsweeps; ++k) {
        uint32_t t = (uint32_t)k;
        if (sampler == 0) {
            n_near += orc_pca_sweep(m, H, W, g, x, tmp, seed, chain, t, NULL);
            memcpy(x, tmp, n);
        } else {
            n_near += orc_gibbs_sweep(m, H, W, g, x, seed, chain, t, gibbs_order, NULL);
        }
        uint32_t idx = 0, mult = 1;
        for (size_t i = 0; i < n; ++i) {
            idx += (uint32_t)x[i] * mult;
            mult *= (uint32_t)m->L;
        }
        hist[idx] += 1.0;
    }
    return n_near;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}
