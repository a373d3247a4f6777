/*
 * prosper_oracle.c -- plain FP64 CPU oracle for the truncated-posterior EM
 * (Expectation Truncation, ET) of three ProSper models: BSC, MCA and GSC.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product library never
 * links, loads or calls it, and it shares no code with the CUDA sources.
 *
 * What it computes (paper: Exarchakis et al., "ProSper", JMLR MLOSS):
 *   - The generative model template of Eq. 1-2: a prior p(s|Theta) and a
 *     noise model p(y|s,Theta) = p(y; f(Theta,s)), with the per-model prior,
 *     noise and superposition f from Table 1 (rows BSC, TSC, DSC, GSC, MCA,
 *     MMCA).  MMCA is MCA with a signed dictionary whose superposition takes,
 *     per pixel, the active component of largest magnitude.
 *     TSC and DSC are linear superpositions like BSC with latents taking
 *     values in a finite set Phi = {0, phi_1, .., phi_m} under a categorical
 *     prior (TSC: Phi = {-1, 0, 1}, zero-mean: p(-1) = p(1) = pi/2).
 *   - EM with truncated posteriors (Sec. 2): for each data point n a set of
 *     H' candidate latents I_n is preselected, the state set K_n holds every
 *     binary pattern over I_n with at most gamma active units (the
 *     BSC_ET(D,H,Hprime,gamma) arguments of Sec. 3), and the posterior is
 *     q_n(s) = p(s,y_n) / sum_{s' in K_n} p(s',y_n) on K_n, zero elsewhere.
 *   - The sufficient statistics of that truncated posterior and the
 *     closed-form M-steps ("Model.step", Sec. 3).
 *
 * The paper defers the per-model equations to its references; every formula
 * below is derived from the model definitions of Eq. 1-2 and Table 1 by
 * textbook Gaussian algebra, written in the plainest form (the log-joint is
 * evaluated from its definition, e.g. ||y - f(s)||^2 with f built per state,
 * and the GSC marginal with a full D x D covariance).  Readings where the
 * paper is silent (selection scores, tie rules, the MCA rho-update) are
 * listed where they are used.
 *
 * Layouts: Y is N x D row-major; W is stored transposed as Wt, H x D
 * row-major (row h is dictionary element W_h, the h-th column of the paper's
 * D x H matrix W).  All arithmetic is double precision.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_BSC = 0, ORC_MCA = 1, ORC_GSC = 2, ORC_TSC = 3, ORC_DSC = 4, ORC_MMCA = 5 };

/* scal[] layout of the aggregated scalar statistics; SC_DSC0 + v holds
 * sum_n sum_h <[s_h = phi_{v+1}]> (TSC/DSC: expected count of each nonzero value) */
enum { SC_F = 0, SC_S1 = 1, SC_YY = 2, SC_N = 3, SC_MCA_R2 = 4, SC_DSC0 = 5, SC_LEN = 8 };

/* theta[] of the oracle: pi, sigma, rho, T, then for DSC the prior
 * probabilities of the m nonzero values (4 .. 4+m-1), m (7) and the values
 * phi_1 .. phi_m (8 .. 8+m-1). */
enum { TH_PI = 0, TH_SIGMA = 1, TH_RHO = 2, TH_T = 3, TH_DSC_P = 4, TH_DSC_M = 7, TH_DSC_V = 8,
       TH_LEN = 12 };
#define MAXV 3   /* nonzero values of a discrete latent */

static const double LOG_2PI = 1.8378770664093454835606594728112;

/* ------------------------------------------------------------------------
 * State set K (Sec. 3: approximation parameters Hprime and gamma).
 * Canonical order: by number of active units, then lexicographic order of
 * the sorted list of active local indices (the order of itertools.combinations).
 * Bit j of a mask is local unit j, i.e. global latent I_n[j].
 * ---------------------------------------------------------------------- */
static double binom(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

int orc_num_states(int Hp, int gamma) {
    double c = 0.0;
    for (int k = 0; k <= gamma && k <= Hp; ++k) c += binom(Hp, k);
    return (int)(c + 0.5);
}

int orc_states(int Hp, int gamma, uint32_t *masks, int cap) {
    int n = 0;
    int idx[32];
    for (int k = 0; k <= gamma && k <= Hp; ++k) {
        for (int i = 0; i < k; ++i) idx[i] = i;
        for (;;) {
            uint32_t m = 0;
            for (int i = 0; i < k; ++i) m |= 1u << idx[i];
            if (n < cap) masks[n] = m;
            ++n;
            /* next combination in lexicographic order */
            int i = k - 1;
            while (i >= 0 && idx[i] == Hp - k + i) --i;
            if (i < 0) break;
            ++idx[i];
            for (int j = i + 1; j < k; ++j) idx[j] = idx[j - 1] + 1;
        }
    }
    return n;
}

/* Discrete latents (TSC, DSC): every pattern of at most gamma nonzero units,
 * each nonzero unit taking one of m values.  Canonical order: by number of
 * nonzero units, then the lexicographic order of their sorted local indices,
 * then the lexicographic order of their value indices (0 .. m-1, in unit
 * order).  vcodes[n] holds the value index of the a-th nonzero unit in bits
 * 2a, 2a+1.  With m = 1 this is the binary order of orc_states. */
int orc_num_states_m(int Hp, int gamma, int m) {
    double c = 0.0, mk = 1.0;
    for (int k = 0; k <= gamma && k <= Hp; ++k) { c += binom(Hp, k) * mk; mk *= m; }
    return (int)(c + 0.5);
}

int orc_states_dsc(int Hp, int gamma, int m, uint32_t *masks, uint32_t *vcodes, int cap) {
    int n = 0;
    int idx[32];
    for (int k = 0; k <= gamma && k <= Hp; ++k) {
        for (int i = 0; i < k; ++i) idx[i] = i;
        for (;;) {
            uint32_t mk = 0;
            for (int i = 0; i < k; ++i) mk |= 1u << idx[i];
            uint32_t nv = 1;
            for (int i = 0; i < k; ++i) nv *= (uint32_t)m;
            for (uint32_t c = 0; c < nv; ++c) {
                /* c in base m, most significant digit = first unit */
                uint32_t code = 0, r = c;
                for (int a = k - 1; a >= 0; --a) { code |= (r % (uint32_t)m) << (2 * a); r /= (uint32_t)m; }
                if (n < cap) { masks[n] = mk; if (vcodes) vcodes[n] = code; }
                ++n;
            }
            int i = k - 1;
            while (i >= 0 && idx[i] == Hp - k + i) --i;
            if (i < 0) break;
            ++idx[i];
            for (int j = i + 1; j < k; ++j) idx[j] = idx[j - 1] + 1;
        }
    }
    return n;
}

static int popcount32(uint32_t m) {
    int c = 0;
    while (m) { c += (int)(m & 1u); m >>= 1; }
    return c;
}

/* ------------------------------------------------------------------------
 * Small dense FP64 linear algebra (textbook Cholesky, Golub & Van Loan 4.2).
 * ---------------------------------------------------------------------- */
/* In place: A (n x n, row-major, symmetric positive definite) -> lower L. */
static int cholesky(double *A, int n) {
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
        if (!(d > 0.0)) return -1;
        double ljj = sqrt(d);
        A[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = s / ljj;
        }
        for (int k = j + 1; k < n; ++k) A[j * n + k] = 0.0;
    }
    return 0;
}

/* Solve L L^T x = b in place (L lower, from cholesky()). */
static void chol_solve(const double *L, int n, double *b) {
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i * n + k] * b[k];
        b[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * b[k];
        b[i] = s / L[i * n + i];
    }
}

/* Solve L v = b in place (forward substitution only). */
static void forward_solve(const double *L, int n, double *b) {
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i * n + k] * b[k];
        b[i] = s / L[i * n + i];
    }
}

/* ------------------------------------------------------------------------
 * Problem description shared by the per-point routines.
 * ---------------------------------------------------------------------- */
typedef struct {
    int model, D, H, Hp, gamma, nK;
    const double *Wt;      /* H x D */
    double pi, sigma, rho; /* sigma = noise standard deviation */
    double T;              /* posterior temperature of deterministic annealing (1 = none) */
    const double *mu, *psi;/* GSC: slab means and variances (H each) */
    const uint32_t *K;     /* nK canonical state masks over local units */
    const uint32_t *V;     /* nK value codes (2 bits per nonzero unit, in unit order) */
    int m;                 /* number of nonzero values (1 for the binary models) */
    double phi[MAXV];      /* the nonzero values (binary models: phi_1 = 1) */
    double lp0, lpv[MAXV]; /* log prior probability of 0 and of each nonzero value */
} problem_t;

/* Per-thread scratch for one data point. */
typedef struct {
    double *score, *ell, *q, *f, *r;     /* H, nK, nK, D, D */
    double *C, *CW, *kappa, *lambda;     /* D*D, D*gamma, nK*Hp, nK*Hp*Hp */
    double *Abar;                        /* MCA: Hp*D expected A_dh */
} scratch_t;

static void scratch_alloc(scratch_t *s, const problem_t *p) {
    int D = p->D, g = p->gamma > 0 ? p->gamma : 1;
    s->score = malloc(sizeof(double) * p->H);
    s->ell = malloc(sizeof(double) * p->nK);
    s->q = malloc(sizeof(double) * p->nK);
    s->f = malloc(sizeof(double) * D);
    s->r = malloc(sizeof(double) * D);
    s->C = p->model == ORC_GSC ? malloc(sizeof(double) * D * D) : NULL;
    s->CW = p->model == ORC_GSC ? malloc(sizeof(double) * D * g) : NULL;
    s->kappa = malloc(sizeof(double) * p->nK * p->Hp);
    s->lambda = malloc(sizeof(double) * p->nK * p->Hp * p->Hp);
    s->Abar = (p->model == ORC_MCA || p->model == ORC_MMCA) ? malloc(sizeof(double) * p->Hp * D) : NULL;
}

static void scratch_free(scratch_t *s) {
    free(s->score); free(s->ell); free(s->q); free(s->f); free(s->r);
    free(s->C); free(s->CW); free(s->kappa); free(s->lambda); free(s->Abar);
}

/* log p(s|Theta) of a binary pattern with k active units out of H:
 * Bernoulli prior (Table 1, BSC and MCA; the spike of GSC's spike-and-slab). */
static double log_prior(const problem_t *p, int k) {
    return k * log(p->pi) + (p->H - k) * log(1.0 - p->pi);
}

/* Categorical prior of a discrete state (Table 1, TSC and DSC): every unit
 * independently 0 with probability pi_0, phi_v with probability pi_v. */
static double log_prior_dsc(const problem_t *p, uint32_t mask, uint32_t vcode) {
    int k = popcount32(mask);
    double l = (p->H - k) * p->lp0;
    for (int a = 0; a < k; ++a) l += p->lpv[(vcode >> (2 * a)) & 3u];
    return l;
}

static int is_discrete(const problem_t *p) { return p->model == ORC_TSC || p->model == ORC_DSC; }
static int is_maxlike(const problem_t *p) { return p->model == ORC_MCA || p->model == ORC_MMCA; }

/* Superposition of the max models at one pixel over the active units gidx[0..k)
 * (Table 1): MCA f_d = max_h W_dh s_h (W >= 0); MMCA f_d = the W_dh of largest
 * |W_dh| among the active units (the first in unit order on a tie in |W|).
 * 0 for the empty state. */
static double superpose_max(const problem_t *p, const int *gidx, int k, int d) {
    double f = 0.0;
    for (int i = 0; i < k; ++i) {
        double w = p->Wt[(size_t)gidx[i] * p->D + d];
        if (i == 0) f = w;
        else if (p->model == ORC_MMCA) f = fabs(w) > fabs(f) ? w : f;
        else f = w > f ? w : f;
    }
    return f;
}

/* Gaussian log-density N(y; m, v I_D) with v = sigma^2, from ||y - m||^2. */
static double log_gauss_iso(int D, double sigma, double r2) {
    double v = sigma * sigma;
    return -0.5 * D * (LOG_2PI + log(v)) - 0.5 * r2 / v;
}

/* ------------------------------------------------------------------------
 * GSC marginal for active set b (global indices gidx[0..k)):
 *   y | b ~ N(W_b mu_b, C_b),  C_b = sigma^2 I_D + W_b Psi_b W_b^T
 * and the Gaussian posterior of the slab values z_b given (b, y):
 *   kappa = mu_b + Psi_b W_b^T C_b^{-1} (y - W_b mu_b)
 *   Lambda = Psi_b - Psi_b W_b^T C_b^{-1} W_b Psi_b
 * (standard conditioning of a joint Gaussian; Table 1 row GSC: linear
 * superposition, Gaussian noise, spike-and-slab prior).  Plain D x D form.
 * Returns log N(y; W_b mu_b, C_b).
 * ---------------------------------------------------------------------- */
static double gsc_marginal(const problem_t *p, scratch_t *s, const double *y,
                           const int *gidx, int k, double *kappa, double *lambda,
                           int ldl) {
    int D = p->D;
    double *C = s->C, *r = s->r, *CW = s->CW;
    double v = p->sigma * p->sigma;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            double c = (i == j) ? v : 0.0;
            for (int a = 0; a < k; ++a) {
                const double *w = p->Wt + (size_t)gidx[a] * D;
                c += w[i] * p->psi[gidx[a]] * w[j];
            }
            C[i * D + j] = c;
        }
    if (cholesky(C, D) != 0) return -INFINITY;
    double logdet = 0.0;
    for (int i = 0; i < D; ++i) logdet += 2.0 * log(C[i * D + i]);
    for (int d = 0; d < D; ++d) {
        double m = 0.0;
        for (int a = 0; a < k; ++a) m += p->Wt[(size_t)gidx[a] * D + d] * p->mu[gidx[a]];
        r[d] = y[d] - m;
    }
    /* quadratic form r^T C^{-1} r = ||L^{-1} r||^2 */
    double *tmp = s->f;
    memcpy(tmp, r, sizeof(double) * D);
    forward_solve(C, D, tmp);
    double quad = 0.0;
    for (int d = 0; d < D; ++d) quad += tmp[d] * tmp[d];
    double logN = -0.5 * D * LOG_2PI - 0.5 * logdet - 0.5 * quad;
    if (kappa) {
        /* Cinv_r = C^{-1} r ; CW[:,a] = C^{-1} W_{b_a} */
        memcpy(tmp, r, sizeof(double) * D);
        chol_solve(C, D, tmp);
        for (int a = 0; a < k; ++a) {
            double *col = CW + (size_t)a * D;
            memcpy(col, p->Wt + (size_t)gidx[a] * D, sizeof(double) * D);
            chol_solve(C, D, col);
        }
        for (int a = 0; a < k; ++a) {
            const double *wa = p->Wt + (size_t)gidx[a] * D;
            double t = 0.0;
            for (int d = 0; d < D; ++d) t += wa[d] * tmp[d];
            kappa[a] = p->mu[gidx[a]] + p->psi[gidx[a]] * t;
            for (int c = 0; c < k; ++c) {
                double u = 0.0;
                for (int d = 0; d < D; ++d) u += wa[d] * CW[(size_t)c * D + d];
                lambda[a * ldl + c] = (a == c ? p->psi[gidx[a]] : 0.0)
                                      - p->psi[gidx[a]] * u * p->psi[gidx[c]];
            }
        }
    }
    return logN;
}

/* ------------------------------------------------------------------------
 * Preselection scores (reading: the paper names Hprime but no score).
 *   BSC: signed normalised projection W_h^T y / ||W_h||.
 *   MCA: sum_d W_dh y_d / sum_d W_dh.
 *   GSC: the singleton log-joint log p(e_h, y).
 * ---------------------------------------------------------------------- */
static void selection_scores(const problem_t *p, scratch_t *s, const double *y) {
    int D = p->D;
    for (int h = 0; h < p->H; ++h) {
        const double *w = p->Wt + (size_t)h * D;
        if (p->model == ORC_BSC || is_discrete(p)) {
            /* BSC: W_h^T y / ||W_h||.  TSC/DSC (reading): the largest normalised
             * projection a nonzero value can reach, sign(phi) W_h^T y / ||W_h||
             * maximised over phi in Phi \ {0}: |.| when Phi has both signs. */
            double pr = 0.0, nn = 0.0;
            for (int d = 0; d < D; ++d) { pr += w[d] * y[d]; nn += w[d] * w[d]; }
            double sc = nn > 0.0 ? pr / sqrt(nn) : 0.0;
            if (is_discrete(p)) {
                int pos = 0, neg = 0;
                for (int v = 0; v < p->m; ++v) { pos |= p->phi[v] > 0.0; neg |= p->phi[v] < 0.0; }
                sc = (pos && neg) ? fabs(sc) : (neg ? -sc : sc);
            }
            s->score[h] = sc;
        } else if (is_maxlike(p)) {
            /* MCA: sum_d W_dh y_d / sum_d W_dh; MMCA (reading, W signed):
             * sum_d W_dh y_d / sum_d |W_dh| */
            double pr = 0.0, sw = 0.0;
            for (int d = 0; d < D; ++d) { pr += w[d] * y[d]; sw += p->model == ORC_MMCA ? fabs(w[d]) : w[d]; }
            s->score[h] = sw > 0.0 ? pr / sw : 0.0;
        } else {
            int g = h;
            s->score[h] = log_prior(p, 1) + gsc_marginal(p, s, y, &g, 1, NULL, NULL, 0);
        }
    }
}

/* Top-Hp by score, exact ties to the lower index; result sorted ascending. */
static void select_top(const problem_t *p, const double *score, int *sel) {
    int H = p->H, Hp = p->Hp;
    char *taken = calloc((size_t)H, 1);
    for (int j = 0; j < Hp; ++j) {
        int best = -1;
        for (int h = 0; h < H; ++h)
            if (!taken[h] && (best < 0 || score[h] > score[best])) best = h;
        taken[best] = 1;
        sel[j] = best;
    }
    free(taken);
    for (int i = 1; i < Hp; ++i)            /* insertion sort, ascending */
        for (int j = i; j > 0 && sel[j - 1] > sel[j]; --j) {
            int t = sel[j]; sel[j] = sel[j - 1]; sel[j - 1] = t;
        }
}

/* ------------------------------------------------------------------------
 * Log-joint log p(s, y | Theta) of state K[kk] over selection sel.
 * ---------------------------------------------------------------------- */
static double log_joint(const problem_t *p, scratch_t *s, const double *y,
                        const int *sel, uint32_t mask, uint32_t vcode, double *kappa,
                        double *lambda) {
    int D = p->D, k = popcount32(mask);
    int gidx[32], a = 0;
    for (int j = 0; j < p->Hp; ++j)
        if (mask & (1u << j)) gidx[a++] = sel[j];
    if (p->model == ORC_GSC)
        return log_prior(p, k) + gsc_marginal(p, s, y, gidx, k, kappa, lambda, p->Hp);
    if (is_discrete(p)) {
        /* f(Theta, s) = W s with s_{gidx[i]} = phi of its value index */
        double r2 = 0.0;
        for (int d = 0; d < D; ++d) {
            double f = 0.0;
            for (int i = 0; i < k; ++i)
                f += p->phi[(vcode >> (2 * i)) & 3u] * p->Wt[(size_t)gidx[i] * D + d];
            r2 += (y[d] - f) * (y[d] - f);
        }
        return log_prior_dsc(p, mask, vcode) + log_gauss_iso(D, p->sigma, r2);
    }
    /* f(Theta, s): BSC linear superposition W s; MCA / MMCA the (magnitude) max */
    for (int d = 0; d < D; ++d) {
        double f = 0.0;
        if (p->model == ORC_BSC)
            for (int i = 0; i < k; ++i) f += p->Wt[(size_t)gidx[i] * D + d];
        else
            f = superpose_max(p, gidx, k, d);
        s->f[d] = f;
    }
    double r2 = 0.0;
    for (int d = 0; d < D; ++d) { double e = y[d] - s->f[d]; r2 += e * e; }
    return log_prior(p, k) + log_gauss_iso(D, p->sigma, r2);
}

/* Per-point results. */
typedef struct {
    int sel[32];
    double logZ, map_p;
    int map_state;
    double smean[32];          /* <s_{I_j}> */
    double ss[32 * 32];        /* <s_{I_i} s_{I_j}> */
    double bmean[32];          /* GSC: <b_{I_j}> */
    double sabs;               /* <|s|> (number of active units) */
    double vcnt[MAXV];         /* TSC/DSC: <number of units with value phi_v> */
    double r2;                 /* MCA: <||y - f(s)||^2> */
} point_t;

/* E-step for one data point: selection, log-joints over K, normalisation,
 * posterior moments (Sec. 2: EM with truncated posteriors). */
static void point_estep(const problem_t *p, scratch_t *s, const double *y,
                        const int *sel_forced, point_t *o) {
    int Hp = p->Hp, nK = p->nK, D = p->D;
    if (sel_forced) {
        for (int j = 0; j < Hp; ++j) o->sel[j] = sel_forced[j];
    } else {
        selection_scores(p, s, y);
        select_top(p, s->score, o->sel);
    }
    double m = -INFINITY;
    int arg = 0;
    for (int kk = 0; kk < nK; ++kk) {
        double *kap = s->kappa + (size_t)kk * Hp, *lam = s->lambda + (size_t)kk * Hp * Hp;
        /* GSC: kappa/lambda are compacted over the active units of the state */
        double l = log_joint(p, s, y, o->sel, p->K[kk], p->V[kk],
                             p->model == ORC_GSC ? kap : NULL,
                             p->model == ORC_GSC ? lam : NULL);
        s->ell[kk] = l;
        if (l > m) { m = l; arg = kk; }      /* first maximum in canonical order */
    }
    /* Deterministic annealing (Sec. 3, LinearAnnealing; reading): the posterior
     * at temperature T is q_T(s) = p(s,y)^(1/T) / sum_{s' in K_n} p(s',y)^(1/T),
     * and the per-point free energy is T log sum_{s in K_n} p(s,y)^(1/T)
     * (= log sum_{K_n} p(s,y) at T = 1).  With m = max_s log p(s,y):
     *   T log sum exp(l/T) = m + T log sum exp((l - m)/T). */
    const double T = p->T;
    double Z = 0.0;
    for (int kk = 0; kk < nK; ++kk) Z += exp((s->ell[kk] - m) / T);
    o->logZ = m + T * log(Z);
    for (int kk = 0; kk < nK; ++kk) s->q[kk] = exp((s->ell[kk] - m) / T) / Z;
    o->map_state = arg;
    o->map_p = s->q[arg];
    memset(o->smean, 0, sizeof(o->smean));
    memset(o->ss, 0, sizeof(o->ss));
    memset(o->bmean, 0, sizeof(o->bmean));
    o->sabs = 0.0;
    o->r2 = 0.0;
    memset(o->vcnt, 0, sizeof(o->vcnt));
    for (int kk = 0; kk < nK; ++kk) {
        uint32_t mask = p->K[kk];
        double q = s->q[kk];
        o->sabs += q * popcount32(mask);
        if (is_discrete(p)) {
            /* <s_i> = sum_s q(s) s_i and <s_i s_j> with the units' values */
            int loc[32], k = 0;
            double val[32];
            for (int j = 0; j < Hp; ++j)
                if (mask & (1u << j)) {
                    int v = (int)((p->V[kk] >> (2 * k)) & 3u);
                    o->vcnt[v] += q;
                    val[k] = p->phi[v];
                    loc[k++] = j;
                }
            for (int a = 0; a < k; ++a) {
                o->smean[loc[a]] += q * val[a];
                for (int c = 0; c < k; ++c) o->ss[loc[a] * 32 + loc[c]] += q * val[a] * val[c];
            }
            continue;
        }
        if (p->model == ORC_GSC) {
            const double *kap = s->kappa + (size_t)kk * Hp, *lam = s->lambda + (size_t)kk * Hp * Hp;
            int loc[32], k = 0;
            for (int j = 0; j < Hp; ++j) if (mask & (1u << j)) loc[k++] = j;
            for (int a = 0; a < k; ++a) {
                o->bmean[loc[a]] += q;
                o->smean[loc[a]] += q * kap[a];
                for (int c = 0; c < k; ++c)
                    o->ss[loc[a] * 32 + loc[c]] += q * (lam[a * Hp + c] + kap[a] * kap[c]);
            }
        } else {
            for (int i = 0; i < Hp; ++i) {
                if (!(mask & (1u << i))) continue;
                o->smean[i] += q;
                for (int j = 0; j < Hp; ++j)
                    if (mask & (1u << j)) o->ss[i * 32 + j] += q;
            }
        }
    }
    if (is_maxlike(p)) {
        /* <||y - f(s)||^2> with the hard max (sigma update, reading R8) and
         * <A_dh> with A_dh(s) = s_h (|W_dh| / Wbar_d(s))^(rho-1),
         * Wbar_d(s) = (sum_{h in s} |W_dh|^rho)^(1/rho)  (rho-smoothed max of
         * the magnitudes; |W| = W for MCA). */
        memset(s->Abar, 0, sizeof(double) * Hp * D);
        for (int kk = 0; kk < nK; ++kk) {
            uint32_t mask = p->K[kk];
            double q = s->q[kk];
            int gidx[32], loc[32], k = 0;
            for (int j = 0; j < Hp; ++j) if (mask & (1u << j)) { loc[k] = j; gidx[k++] = o->sel[j]; }
            double r2 = 0.0;
            for (int d = 0; d < D; ++d) {
                double f = superpose_max(p, gidx, k, d);
                r2 += (y[d] - f) * (y[d] - f);
                if (k == 0) continue;
                /* Wbar = m (sum (|W|/m)^rho)^(1/rho) with m = max |W|: the same
                 * value, without overflow of |W|^rho for large rho */
                double mx = 0.0, sp = 0.0;
                for (int i = 0; i < k; ++i) {
                    double w = fabs(p->Wt[(size_t)gidx[i] * D + d]);
                    mx = w > mx ? w : mx;
                }
                if (!(mx > 0.0)) continue;          /* every active |W_dh| is 0: no factor */
                for (int i = 0; i < k; ++i) sp += pow(fabs(p->Wt[(size_t)gidx[i] * D + d]) / mx, p->rho);
                double wbar = mx * pow(sp, 1.0 / p->rho);
                for (int i = 0; i < k; ++i) {
                    double w = fabs(p->Wt[(size_t)gidx[i] * D + d]);
                    s->Abar[loc[i] * D + d] += q * pow(w / wbar, p->rho - 1.0);
                }
            }
            o->r2 += q * r2;
        }
    }
}

static void problem_init(problem_t *p, int model, int D, int H, int Hp, int gamma,
                         const double *Wt, const double *theta, const double *mu,
                         const double *psi, uint32_t **Kbuf) {
    p->model = model; p->D = D; p->H = H; p->Hp = Hp; p->gamma = gamma;
    p->Wt = Wt; p->pi = theta[TH_PI]; p->sigma = theta[TH_SIGMA]; p->rho = theta[TH_RHO];
    p->T = theta[TH_T] > 0.0 ? theta[TH_T] : 1.0;   /* theta[3] <= 0 selects T = 1 */
    p->mu = mu; p->psi = psi;
    /* value set and categorical prior: binary models phi = {1}, prior pi;
     * TSC phi = {-1, 1} with pi/2 each; DSC from theta */
    p->m = 1; p->phi[0] = 1.0;
    double pv[MAXV] = {p->pi, 0.0, 0.0};
    if (model == ORC_TSC) {
        p->m = 2; p->phi[0] = -1.0; p->phi[1] = 1.0;
        pv[0] = pv[1] = 0.5 * p->pi;
    } else if (model == ORC_DSC) {
        p->m = (int)theta[TH_DSC_M];
        for (int v = 0; v < p->m; ++v) { p->phi[v] = theta[TH_DSC_V + v]; pv[v] = theta[TH_DSC_P + v]; }
    }
    double p0 = 1.0;
    for (int v = 0; v < p->m; ++v) { p0 -= pv[v]; p->lpv[v] = log(pv[v]); }
    p->lp0 = log(p0);
    p->nK = orc_num_states_m(Hp, gamma, p->m);
    *Kbuf = malloc(sizeof(uint32_t) * 2 * (size_t)p->nK);
    orc_states_dsc(Hp, gamma, p->m, *Kbuf, *Kbuf + p->nK, p->nK);
    p->K = *Kbuf;
    p->V = *Kbuf + p->nK;
}

/* ------------------------------------------------------------------------
 * orc_estep: full truncated E-step over N points.
 *
 * Inputs:  Y (N x D), Wt (H x D), theta = {pi, sigma, rho, T}, mu/psi (GSC, H
 *          each; NULL otherwise), sel_in (N x Hp ascending global indices to
 *          use instead of preselection; NULL = preselect).
 * Per-point outputs (each may be NULL): sel (N x Hp), smean (N x Hp),
 *          map_idx (N x gamma, ascending, -1 padded), map_val (N x gamma: the
 *          MAP state's value of each listed unit, 0 padded), map_p (N), logZ (N).
 * Aggregates (each may be NULL; overwritten):
 *          At (H x D): sum_n <s>_n y_n^T (A = sum y <s>^T, transposed)
 *          B  (H x H): sum_n <s s^T>_n
 *          scal[SC_LEN]: F = sum_n log sum_{K_n} p(s,y_n), sum <|s|>,
 *                        sum y^T y, N, MCA sum <||y - f||^2>,
 *                        TSC/DSC sum <count of value phi_v> (SC_DSC0 + v)
 *          gsc (3H): sum <b_h>, sum <s_h>, sum <s_h^2>
 *          mca (2 H D): sum <A_dh> y_d, sum <A_dh> (both H x D)
 * ---------------------------------------------------------------------- */
int orc_estep(int model, int64_t N, int D, int H, int Hp, int gamma,
              const double *Y, const double *Wt, const double *theta,
              const double *mu, const double *psi, const int32_t *sel_in,
              int32_t *sel, double *smean, int32_t *map_idx, double *map_val,
              double *map_p, double *logZ, double *At, double *B, double *scal,
              double *gsc, double *mca, int nthreads) {
    if (Hp < 1 || Hp > 32 || Hp > H || gamma < 0 || gamma > Hp) return -1;
    problem_t p;
    uint32_t *Kbuf;
    problem_init(&p, model, D, H, Hp, gamma, Wt, theta, mu, psi, &Kbuf);
    if (At) memset(At, 0, sizeof(double) * H * D);
    if (B) memset(B, 0, sizeof(double) * H * H);
    if (scal) memset(scal, 0, sizeof(double) * SC_LEN);
    if (gsc) memset(gsc, 0, sizeof(double) * 3 * H);
    if (mca) memset(mca, 0, sizeof(double) * 2 * H * D);
    int nt = 1;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    /* per-thread partial sums, combined in thread order at the end */
    double **pAt = calloc(nt, sizeof(double *)), **pB = calloc(nt, sizeof(double *));
    double **pS = calloc(nt, sizeof(double *)), **pG = calloc(nt, sizeof(double *));
    double **pM = calloc(nt, sizeof(double *));
#pragma omp parallel num_threads(nt)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        scratch_t s;
        scratch_alloc(&s, &p);
        double *lAt = At ? calloc((size_t)H * D, sizeof(double)) : NULL;
        double *lB = B ? calloc((size_t)H * H, sizeof(double)) : NULL;
        double *lS = calloc(SC_LEN, sizeof(double));
        double *lG = gsc ? calloc((size_t)3 * H, sizeof(double)) : NULL;
        double *lM = mca ? calloc((size_t)2 * H * D, sizeof(double)) : NULL;
        point_t o;
#pragma omp for schedule(static)
        for (int64_t n = 0; n < N; ++n) {
            const double *y = Y + (size_t)n * D;
            point_estep(&p, &s, y, sel_in ? (const int *)(sel_in + (size_t)n * Hp) : NULL, &o);
            if (sel) for (int j = 0; j < Hp; ++j) sel[(size_t)n * Hp + j] = o.sel[j];
            if (smean) for (int j = 0; j < Hp; ++j) smean[(size_t)n * Hp + j] = o.smean[j];
            if (map_idx || map_val) {
                uint32_t mk = p.K[o.map_state], vc = p.V[o.map_state];
                int a = 0;
                for (int j = 0; j < Hp; ++j)
                    if (mk & (1u << j)) {
                        if (map_idx) map_idx[(size_t)n * gamma + a] = o.sel[j];
                        if (map_val) map_val[(size_t)n * gamma + a] = p.phi[(vc >> (2 * a)) & 3u];
                        ++a;
                    }
                for (; a < gamma; ++a) {
                    if (map_idx) map_idx[(size_t)n * gamma + a] = -1;
                    if (map_val) map_val[(size_t)n * gamma + a] = 0.0;
                }
            }
            if (map_p) map_p[n] = o.map_p;
            if (logZ) logZ[n] = o.logZ;
            double yy = 0.0;
            for (int d = 0; d < D; ++d) yy += y[d] * y[d];
            lS[SC_F] += o.logZ; lS[SC_S1] += o.sabs; lS[SC_YY] += yy; lS[SC_N] += 1.0;
            lS[SC_MCA_R2] += o.r2;
            if (is_discrete(&p)) for (int v = 0; v < p.m; ++v) lS[SC_DSC0 + v] += o.vcnt[v];
            if (lAt) for (int j = 0; j < Hp; ++j) {
                double e = o.smean[j];
                double *row = lAt + (size_t)o.sel[j] * D;
                for (int d = 0; d < D; ++d) row[d] += e * y[d];
            }
            if (lB) for (int i = 0; i < Hp; ++i) for (int j = 0; j < Hp; ++j)
                lB[(size_t)o.sel[i] * H + o.sel[j]] += o.ss[i * 32 + j];
            if (lG) for (int j = 0; j < Hp; ++j) {
                int h = o.sel[j];
                lG[h] += o.bmean[j]; lG[H + h] += o.smean[j]; lG[2 * H + h] += o.ss[j * 32 + j];
            }
            if (lM) for (int j = 0; j < Hp; ++j) {
                int h = o.sel[j];
                for (int d = 0; d < D; ++d) {
                    lM[(size_t)h * D + d] += s.Abar[j * D + d] * y[d];
                    lM[(size_t)H * D + (size_t)h * D + d] += s.Abar[j * D + d];
                }
            }
        }
        pAt[t] = lAt; pB[t] = lB; pS[t] = lS; pG[t] = lG; pM[t] = lM;
        scratch_free(&s);
    }
    for (int t = 0; t < nt; ++t) {
        if (At && pAt[t]) for (size_t i = 0; i < (size_t)H * D; ++i) At[i] += pAt[t][i];
        if (B && pB[t]) for (size_t i = 0; i < (size_t)H * H; ++i) B[i] += pB[t][i];
        if (scal && pS[t]) for (int i = 0; i < SC_LEN; ++i) scal[i] += pS[t][i];
        if (gsc && pG[t]) for (int i = 0; i < 3 * H; ++i) gsc[i] += pG[t][i];
        if (mca && pM[t]) for (size_t i = 0; i < (size_t)2 * H * D; ++i) mca[i] += pM[t][i];
        free(pAt[t]); free(pB[t]); free(pS[t]); free(pG[t]); free(pM[t]);
    }
    free(pAt); free(pB); free(pS); free(pG); free(pM);
    free(Kbuf);
    return 0;
}

/* ------------------------------------------------------------------------
 * ET's data-point cut (reading of the ET variant the paper's references
 * describe; Sec. 2 only names truncated posteriors):
 *   N_cut = floor(N P_pi(|s| <= gamma)),  P_pi(|s| <= gamma) =
 *           sum_{k <= gamma} C(H,k) pi^k (1 - pi)^(H - k)
 * (the expected number of points generated by at most gamma causes), and the
 * M-step uses the points whose log sum_{K_n} p(s, y_n) reaches the N_cut-th
 * largest value (every point tied with it is kept).  Their sum<|s|> is biased
 * towards few causes, so pi is corrected by H pi / E_pi[|s| : |s| <= gamma].
 * ---------------------------------------------------------------------- */
static double binom_pmf_ratio_sum(int H, int gamma, double pi, double *mean_trunc) {
    /* w_k = C(H,k) pi^k (1-pi)^(H-k) / (1-pi)^H = C(H,k) (pi/(1-pi))^k */
    double w = 1.0, sw = 0.0, skw = 0.0;
    for (int k = 0; k <= gamma && k <= H; ++k) {
        sw += w;
        skw += k * w;
        w *= (double)(H - k) / (k + 1) * pi / (1.0 - pi);
    }
    if (mean_trunc) *mean_trunc = skw / sw;
    return sw;
}

/* P_pi(|s| <= gamma) */
double orc_trunc_prob(int H, int gamma, double pi) {
    if (gamma >= H) return 1.0;                  /* every pattern is kept */
    return binom_pmf_ratio_sum(H, gamma, pi, NULL) * exp(H * log1p(-pi));
}

int64_t orc_cut_size(int64_t N, int H, int gamma, double pi) {
    int64_t n = (int64_t)floor((double)N * orc_trunc_prob(H, gamma, pi));
    if (n < 1) n = 1;
    return n > N ? N : n;
}

/* H pi / E_pi[|s| : |s| <= gamma] (1 when gamma >= H: no truncation) */
double orc_pi_correction(int H, int gamma, double pi) {
    if (gamma >= H) return 1.0;
    double m;
    binom_pmf_ratio_sum(H, gamma, pi, &m);
    return m > 0.0 ? H * pi / m : 1.0;
}

/* keep[n] = 1 for the points whose logZ reaches the ncut-th largest value. */
int orc_cut_keep(int64_t N, const double *logZ, int64_t ncut, uint8_t *keep) {
    double *v = malloc(sizeof(double) * (size_t)N);
    memcpy(v, logZ, sizeof(double) * (size_t)N);
    /* the ncut-th largest by a plain selection sort of the top ncut (tests only) */
    for (int64_t i = 0; i < ncut && i < N; ++i) {
        int64_t b = i;
        for (int64_t j = i + 1; j < N; ++j) if (v[j] > v[b]) b = j;
        double t = v[i]; v[i] = v[b]; v[b] = t;
    }
    const double thr = v[(ncut < N ? ncut : N) - 1];
    free(v);
    int64_t kept = 0;
    for (int64_t n = 0; n < N; ++n) { keep[n] = logZ[n] >= thr; kept += keep[n]; }
    return (int)kept;
}

/* ------------------------------------------------------------------------
 * orc_posterior: the full truncated posterior of ONE data point, for tests.
 * Outputs: sel (Hp), masks (nK), vcodes (nK, TSC/DSC value codes; may be
 * NULL), ell (nK log-joints), q (nK),
 * kappa (nK x Hp) and lambda (nK x Hp x Hp) for GSC (compacted over the
 * active units of each state; may be NULL).  Returns nK.
 * ---------------------------------------------------------------------- */
int orc_posterior(int model, int D, int H, int Hp, int gamma, const double *y,
                  const double *Wt, const double *theta, const double *mu,
                  const double *psi, const int32_t *sel_in, int32_t *sel,
                  uint32_t *masks, uint32_t *vcodes, double *ell, double *q,
                  double *kappa, double *lambda, double *scores) {
    if (Hp < 1 || Hp > 32 || Hp > H || gamma < 0 || gamma > Hp) return -1;
    problem_t p;
    uint32_t *Kbuf;
    problem_init(&p, model, D, H, Hp, gamma, Wt, theta, mu, psi, &Kbuf);
    scratch_t s;
    scratch_alloc(&s, &p);
    point_t o;
    selection_scores(&p, &s, y);
    if (scores) memcpy(scores, s.score, sizeof(double) * H);
    point_estep(&p, &s, y, (const int *)sel_in, &o);
    for (int j = 0; j < Hp; ++j) sel[j] = o.sel[j];
    for (int kk = 0; kk < p.nK; ++kk) {
        masks[kk] = p.K[kk];
        if (vcodes) vcodes[kk] = p.V[kk];
        ell[kk] = s.ell[kk];
        q[kk] = s.q[kk];
    }
    if (kappa) memcpy(kappa, s.kappa, sizeof(double) * p.nK * Hp);
    if (lambda) memcpy(lambda, s.lambda, sizeof(double) * p.nK * Hp * Hp);
    int nK = p.nK;
    scratch_free(&s);
    free(Kbuf);
    return nK;
}

/* Selection scores of one point (tests of the preselection rule). */
int orc_scores(int model, int D, int H, const double *y, const double *Wt,
               const double *theta, const double *mu, const double *psi,
               double *scores) {
    problem_t p;
    uint32_t *Kbuf;
    problem_init(&p, model, D, H, 1, 0, Wt, theta, mu, psi, &Kbuf);
    scratch_t s;
    scratch_alloc(&s, &p);
    selection_scores(&p, &s, y);
    memcpy(scores, s.score, sizeof(double) * H);
    scratch_free(&s);
    free(Kbuf);
    return 0;
}

/* ------------------------------------------------------------------------
 * orc_mstep: closed-form M-step (Sec. 3, Model.step; the prior and noise
 * parameters are learned as well as W, Sec. 1).
 *
 * BSC, TSC, DSC, GSC (maximise the expected log-joint Q; exact argmax):
 *   W = A B^{-1}  ->  Wt = B^{-1} At   (FP64 Cholesky)
 *   pi = sum<|s|> / (N H)
 *   sigma^2 = (sum y^T y - 2 tr(W^T A) + tr(W^T W B)) / (N D)   (new W)
 *   GSC: mu_h = sum<s_h>/sum<b_h>,
 *        psi_h = (sum<s_h^2> - 2 mu_h sum<s_h> + mu_h^2 sum<b_h>)/sum<b_h>
 * MCA (rho-smoothed max update, reading):
 *   W_dh = sum<A_dh> y_d / sum<A_dh>  (kept when the denominator is 0),
 *   clamped to >= 1e-6; pi as above; sigma^2 = sum<||y - f(s)||^2>/(N D).
 * A unit whose B_hh <= 1e-9 N (never active) keeps its old W_h (and mu, psi);
 * the system decouples exactly for such a unit.  The active block of B gets
 * a ridge of 1e-9 tr(B)/H on its diagonal before the Cholesky.
 * Outputs overwrite Wt (H x D), theta (pi, sigma), mu, psi.
 * ---------------------------------------------------------------------- */
int orc_mstep(int model, int D, int H, double Ntot, const double *At,
              const double *B, const double *scal, const double *gsc,
              const double *mca, double *Wt, double *theta, double *mu,
              double *psi) {
    if (model == ORC_MCA || model == ORC_MMCA) {
        /* MCA keeps W >= 1e-6 (its powers need W > 0); MMCA's W is signed */
        for (int h = 0; h < H; ++h)
            for (int d = 0; d < D; ++d) {
                double num = mca[(size_t)h * D + d], den = mca[(size_t)H * D + (size_t)h * D + d];
                if (den > 0.0) {
                    double w = num / den;
                    Wt[(size_t)h * D + d] = (model == ORC_MCA && w < 1e-6) ? 1e-6 : w;
                }
            }
        theta[0] = scal[SC_S1] / (Ntot * H);
        theta[1] = sqrt(scal[SC_MCA_R2] / (Ntot * D));
        return 0;
    }
    double *Bm = malloc(sizeof(double) * H * H);
    double *X = malloc(sizeof(double) * H * D);
    double trB = 0.0;
    for (int h = 0; h < H; ++h) trB += B[(size_t)h * H + h];
    double ridge = 1e-9 * trB / H;
    char *active = malloc((size_t)H);
    for (int h = 0; h < H; ++h) active[h] = B[(size_t)h * H + h] > 1e-9 * Ntot;
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < H; ++j) {
            double b;
            if (active[i] && active[j]) b = B[(size_t)i * H + j] + (i == j ? ridge : 0.0);
            else b = (i == j) ? 1.0 : 0.0;
            Bm[(size_t)i * H + j] = b;
        }
    for (int h = 0; h < H; ++h)
        for (int d = 0; d < D; ++d)
            X[(size_t)h * D + d] = active[h] ? At[(size_t)h * D + d] : Wt[(size_t)h * D + d];
    if (cholesky(Bm, H) != 0) { free(Bm); free(X); free(active); return -2; }
    double *col = malloc(sizeof(double) * H);
    for (int d = 0; d < D; ++d) {
        for (int h = 0; h < H; ++h) col[h] = X[(size_t)h * D + d];
        chol_solve(Bm, H, col);
        for (int h = 0; h < H; ++h) Wt[(size_t)h * D + d] = col[h];
    }
    free(col);
    /* sigma^2 with the new W */
    double t1 = 0.0, t2 = 0.0;
    for (size_t i = 0; i < (size_t)H * D; ++i) t1 += Wt[i] * At[i];
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < H; ++j) {
            double g = 0.0;
            for (int d = 0; d < D; ++d) g += Wt[(size_t)i * D + d] * Wt[(size_t)j * D + d];
            t2 += g * B[(size_t)i * H + j];
        }
    double s2 = (scal[SC_YY] - 2.0 * t1 + t2) / (Ntot * D);
    /* Bernoulli (BSC, GSC spike) and zero-mean ternary (TSC: p(+-1) = pi/2):
     * pi = expected fraction of nonzero units.  DSC: each nonzero value's
     * probability = its expected fraction (the categorical argmax of Q). */
    theta[TH_PI] = scal[SC_S1] / (Ntot * H);
    theta[TH_SIGMA] = sqrt(s2 > 0.0 ? s2 : 0.0);
    if (model == ORC_DSC)
        for (int v = 0; v < (int)theta[TH_DSC_M]; ++v) theta[TH_DSC_P + v] = scal[SC_DSC0 + v] / (Ntot * H);
    if (model == ORC_GSC) {
        for (int h = 0; h < H; ++h) {
            double sb = gsc[h], ss = gsc[H + h], ss2 = gsc[2 * H + h];
            if (!(sb > 1e-9 * Ntot)) continue;
            double m = ss / sb;
            double v = (ss2 - 2.0 * m * ss + m * m * sb) / sb;
            mu[h] = m;
            psi[h] = v > 1e-8 ? v : 1e-8;
        }
    }
    free(Bm); free(X); free(active);
    return 0;
}
