/*
 * ndgsbp_oracle.c -- plain FP64 CPU oracle for non-disjoint group shuffled belief propagation
 * (NDGSBP) decoding of LDPC codes, written from Hsu, Chang, Su and Weng, "A Non-Disjoint Group
 * Shuffled Decoding for LDPC Codes".
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously correct reference that the CUDA decoder
 * is compared against.  It shares no code, header, table or helper with the CUDA library and
 * neither side loads the other.  Only the test suite, the package smoke check and the CPU
 * baseline of the benchmark load it.
 *
 * What is here, in the paper's order:
 *   oracle_group_sizes     the size relation G*N_G - (G-1)*N_G*r = M (Sec. II-A), in integers
 *   oracle_groups          Step 1, grouping check nodes (Sec. II-C)
 *   oracle_ndgsbp_decode   Steps 2-4 (Sec. II-C): CN update Eq. (1), VN update Eq. (2), total
 *                          LLR Eq. (3), hard decision and syndrome stop; every edge message is
 *                          stored in both directions, as the paper writes them
 *   oracle_flood_decode    textbook flooding sum-product (the G = 1 reduction)
 *   oracle_layered_decode  textbook row-serial layered BP (the N_G = 1, r = 0 reduction)
 *   oracle_group_posterior_decode  textbook group-shuffled BP in posterior form (a second
 *                          formulation of Step 2 for any groups, overlapping or not)
 *   oracle_philox4x32_10   Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
 *                          SC'11) and oracle_awgn_llr, the BPSK/AWGN channel of Sec. II-C
 *   oracle_budget_iters    the equal-complexity iteration allowance of Sec. IV
 *
 * Readings of points the paper leaves open (each is also listed in the design notes):
 *   - N_G = ceil(M / (G - (G-1) r)); overlap o = round-half-up(r N_G); the M - N_G CNs after the
 *     first group are split over groups 2..G as evenly as possible, larger shares first.
 *   - "randomly" in Step 1 is SplitMix64 driving a forward Fisher-Yates draw; the r N_G CNs a
 *     group takes from its predecessor are the last o CNs of that predecessor in draw order,
 *     which is a uniformly random subset of G_{g-1} \ G_{g-2} when o <= |G_{g-1} \ G_{g-2}|.
 *   - groups are built once and kept for every iteration (a per-iteration redraw is available
 *     in the decoder through several groupings cycled by iteration).
 *   - messages start at L_{m->n} = 0 and L_{n->m} = L_n.
 *   - VN->CN inputs to Eq. (1) and its outputs are clipped to |x| <= llr_max (llr_max <= 0
 *     disables clipping); |product| is held below 1 - 1e-15 so atanh stays finite.
 *   - a tie L_total = 0 decides bit 0; the stop test runs once per full iteration.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_EINFEASIBLE (-2)
#define ORACLE_ENOMEM (-3)

/* ------------------------------------------------------------------------------------------
 * SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number generators", 2014).
 * ---------------------------------------------------------------------------------------- */
static uint64_t splitmix64_next(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------------------------------------
 * Group sizes (Sec. II-A: G N_G - (G-1) N_G r = M).
 *   linear groups:  N_G = ceil(M / (G - (G-1) r)), o = round-half-up(r N_G),
 *                   fresh[0] = N_G, fresh[1..G-1] share M - N_G as evenly as possible.
 *   cyclic groups:  the G windows tile a ring of M units with stride s = M / G (must divide);
 *                   o = round-half-up(r s / (1 - r)), N_G = s + o, fresh[g] = s.
 * Returns 0 or a negative error.
 * ---------------------------------------------------------------------------------------- */
int oracle_group_sizes(int M, int G, double r, int cyclic, int *NG_out, int *o_out, int *fresh) {
    if (M < 1 || G < 1 || G > M || !(r >= 0.0) || !(r < 1.0)) return ORACLE_EINVAL;
    int NG, o;
    if (cyclic) {
        if (M % G) return ORACLE_EINFEASIBLE;
        int s = M / G;
        o = (int)floor(r * s / (1.0 - r) + 0.5 + 1e-9);
        NG = s + o;
        if (NG > M) return ORACLE_EINFEASIBLE;
        for (int g = 0; g < G; ++g) fresh[g] = s;
    } else {
        double x = (double)M / ((double)G - (double)(G - 1) * r);
        NG = (int)ceil(x - 1e-9 * x);
        if (NG > M) NG = M;
        if (G == 1) NG = M;
        o = (G == 1) ? 0 : (int)floor(r * NG + 0.5 + 1e-9);
        fresh[0] = NG;
        if (G > 1) {
            int rest = M - NG;
            int share = rest / (G - 1), extra = rest % (G - 1);
            for (int g = 1; g < G; ++g) {
                fresh[g] = share + ((g - 1) < extra ? 1 : 0);
                if (fresh[g] < 1) return ORACLE_EINFEASIBLE;
            }
        }
        if (o > NG) return ORACLE_EINFEASIBLE;
    }
    *NG_out = NG;
    *o_out = o;
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------------------------
 * Step 1: grouping check nodes (Sec. II-C).
 *
 * Units are single CNs (unit = 1) or layers of `unit` consecutive CNs (QC codes).  The set U of
 * unused units starts full.  G_1 takes N_G units drawn at random from U; each later G_g takes
 * the last o units of G_{g-1} (its overlap with the previous group) followed by fresh[g] units
 * drawn at random from what is left of U.  A draw of k units is k steps of a forward
 * Fisher-Yates shuffle of U driven by SplitMix64(seed): at step i the unit at position i is
 * swapped with the one at position i + (next() mod (|U| - i)).  With `natural` set, the draw
 * takes units in index order instead (no shuffle).  Cyclic grouping draws the whole order once
 * and takes window g as units (g s + j) mod M_u, j < N_G.
 *
 * Output: grp_ptr[G+1] and grp_cn[] (CN indices, each group's units in order, each unit's CNs
 * ascending).  Returns the number of entries written or a negative error.
 * ---------------------------------------------------------------------------------------- */
int oracle_groups(int M, int unit, int G, double r, uint64_t seed, int cyclic, int natural,
                  int *grp_ptr, int *grp_cn, int cap) {
    if (unit < 1 || M % unit) return ORACLE_EINVAL;
    int Mu = M / unit;
    int *fresh = (int *)malloc(sizeof(int) * (size_t)G);
    int *U = (int *)malloc(sizeof(int) * (size_t)Mu);
    int *units = NULL;
    if (!fresh || !U) { free(fresh); free(U); return ORACLE_ENOMEM; }
    int NG, o;
    int rc = oracle_group_sizes(Mu, G, r, cyclic, &NG, &o, fresh);
    if (rc) { free(fresh); free(U); return rc; }
    for (int i = 0; i < Mu; ++i) U[i] = i;
    uint64_t state = seed;
    int pos = 0; /* units U[0..pos) have been drawn, in draw order */
#define DRAW(k)                                                                   \
    for (int _i = 0; _i < (k); ++_i, ++pos) {                                     \
        if (!natural) {                                                           \
            int _j = pos + (int)(splitmix64_next(&state) % (uint64_t)(Mu - pos)); \
            int _t = U[pos]; U[pos] = U[_j]; U[_j] = _t;                          \
        }                                                                         \
    }
    /* unit lists per group */
    int total_units = 0;
    for (int g = 0; g < G; ++g) total_units += (g == 0 ? NG : (cyclic ? NG : o + fresh[g]));
    units = (int *)malloc(sizeof(int) * (size_t)total_units);
    if (!units) { free(fresh); free(U); return ORACLE_ENOMEM; }
    int *gstart = (int *)malloc(sizeof(int) * (size_t)(G + 1));
    int w = 0;
    if (cyclic) {
        DRAW(Mu);
        int s = Mu / G;
        for (int g = 0; g < G; ++g) {
            gstart[g] = w;
            for (int j = 0; j < NG; ++j) units[w++] = U[(g * s + j) % Mu];
        }
    } else {
        gstart[0] = 0;
        DRAW(NG);
        for (int j = 0; j < NG; ++j) units[w++] = U[j];
        for (int g = 1; g < G; ++g) {
            gstart[g] = w;
            int prev_begin = gstart[g - 1], prev_len = gstart[g] - gstart[g - 1];
            for (int j = prev_len - o; j < prev_len; ++j) units[w++] = units[prev_begin + j];
            int first_new = pos;
            DRAW(fresh[g]);
            for (int j = first_new; j < pos; ++j) units[w++] = U[j];
        }
    }
    gstart[G] = w;
#undef DRAW
    int need = w * unit;
    if (need > cap) { free(fresh); free(U); free(units); free(gstart); return ORACLE_EINVAL; }
    int e = 0;
    for (int g = 0; g < G; ++g) {
        grp_ptr[g] = e;
        for (int j = gstart[g]; j < gstart[g + 1]; ++j)
            for (int c = 0; c < unit; ++c) grp_cn[e++] = units[j] * unit + c;
    }
    grp_ptr[G] = e;
    free(fresh); free(U); free(units); free(gstart);
    return e;
}

/* Equal-complexity iteration allowance of Sec. IV: M I_max / (M + (G-1) N_G r), real-valued as
 * printed (the paper's example gives 627 for M = 252, G = 12, N_G = 34, r = 0.4, I_max = 1000),
 * truncated to an integer. */
int oracle_budget_iters(int M, int G, int NG, double r, int imax) {
    double v = (double)M * imax / ((double)M + (double)(G - 1) * NG * r);
    return (int)floor(v + 1e-9);
}

/* ------------------------------------------------------------------------------------------
 * Shared decoder plumbing: a column (VN) view of H and a thread pool over frames.
 * ---------------------------------------------------------------------------------------- */
struct Work;
typedef struct {
    int M, N, E;
    const int *row_ptr, *col_idx;
    int *col_ptr;   /* [N+1] */
    int *col_edge;  /* [E]   edge ids (CSR positions) of VN n, ascending CN order */
    int G;          /* groups per iteration */
    const int *grp_ptr, *grp_cn;
    int n_groupings;          /* > 1: grouping l % n_groupings is used in iteration l */
    const double *llr;
    long n_frames;
    int max_iter;
    double llr_max;
    int early_stop;
    int stop_after_subiters;
    uint8_t *hard;
    int *iters;
    uint8_t *synd_ok;
    double *total;
    double *c2v_out;
    int max_deg_row, max_deg_col;
    int *edge_row;  /* [E] CN of each edge (vertical schedule only; NULL otherwise) */
    long next_frame;
    pthread_mutex_t lock;
    void (*frame_fn)(const void *ctx, long f, struct Work *w);
} Ctx;

/* Per-thread scratch for one frame at a time. */
typedef struct Work {
    double *a, *b;      /* [E] each: the two edge-message arrays */
    double *tot;        /* [N] */
    double *th;         /* [max row degree] */
    uint8_t *d, *mark;  /* [N] each */
    int *touched;       /* [N] */
} Work;

static int build_columns(Ctx *c) {
    c->col_ptr = (int *)calloc((size_t)c->N + 1, sizeof(int));
    c->col_edge = (int *)malloc(sizeof(int) * (size_t)(c->E > 0 ? c->E : 1));
    if (!c->col_ptr || !c->col_edge) return ORACLE_ENOMEM;
    for (int e = 0; e < c->E; ++e) c->col_ptr[c->col_idx[e] + 1]++;
    for (int n = 0; n < c->N; ++n) c->col_ptr[n + 1] += c->col_ptr[n];
    int *fill = (int *)malloc(sizeof(int) * (size_t)c->N);
    if (!fill) return ORACLE_ENOMEM;
    memcpy(fill, c->col_ptr, sizeof(int) * (size_t)c->N);
    for (int m = 0; m < c->M; ++m)
        for (int e = c->row_ptr[m]; e < c->row_ptr[m + 1]; ++e) c->col_edge[fill[c->col_idx[e]]++] = e;
    free(fill);
    c->max_deg_row = 0;
    for (int m = 0; m < c->M; ++m) {
        int d = c->row_ptr[m + 1] - c->row_ptr[m];
        if (d > c->max_deg_row) c->max_deg_row = d;
    }
    c->max_deg_col = 0;
    for (int n = 0; n < c->N; ++n) {
        int d = c->col_ptr[n + 1] - c->col_ptr[n];
        if (d > c->max_deg_col) c->max_deg_col = d;
    }
    return ORACLE_OK;
}

static double clip(double x, double lim) {
    if (lim <= 0.0) return x;
    if (x > lim) return lim;
    if (x < -lim) return -lim;
    return x;
}

/* Eq. (1) for one CN m: L_{m->n} = 2 atanh( prod_{n' in N(m)\n} tanh(L_{n'->m} / 2) ), the product
 * taken directly over the other edges of the row (no division, no log-domain trick).  `th` is
 * scratch of the row's degree. */
static void cn_update_eq1(const Ctx *c, int m, const double *v2c, double *c2v, double *th) {
    int b = c->row_ptr[m], d = c->row_ptr[m + 1] - b;
    for (int k = 0; k < d; ++k) th[k] = tanh(0.5 * clip(v2c[b + k], c->llr_max));
    for (int k = 0; k < d; ++k) {
        double prod = 1.0;
        for (int j = 0; j < d; ++j)
            if (j != k) prod *= th[j];
        const double lim = 1.0 - 1e-15;
        if (prod > lim) prod = lim;
        if (prod < -lim) prod = -lim;
        c2v[b + k] = clip(2.0 * atanh(prod), c->llr_max);
    }
}

/* Eq. (3) and Step 4: total LLR, hard decision (d_n = 0 iff total >= 0) and syndrome. */
static int total_and_syndrome(const Ctx *c, const double *L, const double *c2v, double *tot, uint8_t *d) {
    for (int n = 0; n < c->N; ++n) {
        double s = L[n];
        for (int i = c->col_ptr[n]; i < c->col_ptr[n + 1]; ++i) s += c2v[c->col_edge[i]];
        tot[n] = s;
        d[n] = (s < 0.0) ? 1 : 0;
    }
    for (int m = 0; m < c->M; ++m) {
        int p = 0;
        for (int e = c->row_ptr[m]; e < c->row_ptr[m + 1]; ++e) p ^= d[c->col_idx[e]];
        if (p) return 0;
    }
    return 1;
}

static void write_outputs(const Ctx *c, long f, int l, int ok, const double *tot, const uint8_t *d,
                          const double *c2v) {
    memcpy(c->hard + (size_t)f * c->N, d, (size_t)c->N);
    c->iters[f] = l;
    c->synd_ok[f] = (uint8_t)ok;
    if (c->total) memcpy(c->total + (size_t)f * c->N, tot, sizeof(double) * (size_t)c->N);
    if (c->c2v_out) memcpy(c->c2v_out + (size_t)f * c->E, c2v, sizeof(double) * (size_t)c->E);
}

/* ------------------------------------------------------------------------------------------
 * NDGSBP, Steps 2-4 of Sec. II-C, one frame.
 * ---------------------------------------------------------------------------------------- */
static void ndgsbp_frame(const void *vctx, long f, Work *w) {
    const Ctx *c = (const Ctx *)vctx;
    const int E = c->E, N = c->N;
    const double *L = c->llr + (size_t)f * N;
    double *v2c = w->a, *c2v = w->b, *tot = w->tot, *th = w->th;
    uint8_t *d = w->d, *mark = w->mark;
    int *touched = w->touched;
    /* Initialisation: L_{n->m} = L_n, L_{m->n} = 0 */
    for (int e = 0; e < E; ++e) v2c[e] = L[c->col_idx[e]];
    for (int e = 0; e < E; ++e) c2v[e] = 0.0;
    memset(mark, 0, (size_t)N);
    int sub = 0, l = 1, ok = 0;
    for (l = 1;; ++l) {
        int gi = (c->n_groupings > 1) ? ((l - 1) % c->n_groupings) : 0;
        const int *gp = c->grp_ptr + (size_t)gi * (c->G + 1);
        for (int g = 0; g < c->G; ++g) {
            /* Step 2 a): CN update, Eq. (1), for every m in G_g.  The VN->CN messages are not
             * written during this loop, so every CN of the group reads them as they stood at
             * the start of the sub-iteration (the CNs of a group are updated in parallel). */
            for (int i = gp[g]; i < gp[g + 1]; ++i) cn_update_eq1(c, c->grp_cn[i], v2c, c2v, th);
            /* Step 2 b): VN update, Eq. (2), for every n in the union of N(m), m in G_g, and
             * every m in M(n): L_{n->m} = L_n + sum over m' in M(n)\m of L_{m'->n}. */
            int nt = 0;
            for (int i = gp[g]; i < gp[g + 1]; ++i) {
                int m = c->grp_cn[i];
                for (int e = c->row_ptr[m]; e < c->row_ptr[m + 1]; ++e) {
                    int n = c->col_idx[e];
                    if (!mark[n]) { mark[n] = 1; touched[nt++] = n; }
                }
            }
            for (int t = 0; t < nt; ++t) {
                int n = touched[t];
                mark[n] = 0;
                for (int i = c->col_ptr[n]; i < c->col_ptr[n + 1]; ++i) {
                    int e = c->col_edge[i];
                    double s = L[n];
                    for (int j = c->col_ptr[n]; j < c->col_ptr[n + 1]; ++j)
                        if (j != i) s += c2v[c->col_edge[j]];
                    v2c[e] = s;
                }
            }
            if (c->stop_after_subiters > 0 && ++sub == c->stop_after_subiters) {
                ok = total_and_syndrome(c, L, c2v, tot, d);
                write_outputs(c, f, l, ok, tot, d, c2v);
                return;
            }
        }
        /* Step 3: Eq. (3); Step 4: hard decision and stopping test */
        ok = total_and_syndrome(c, L, c2v, tot, d);
        if ((ok && c->early_stop) || l >= c->max_iter) break;
    }
    write_outputs(c, f, l, ok, tot, d, c2v);
}

/* ------------------------------------------------------------------------------------------
 * Textbook flooding sum-product (all CNs, then all VNs), posterior form: the VN->CN message is
 * the total LLR minus the incoming message on the same edge.  Independent of the group code
 * above; the G = 1 NDGSBP schedule must reproduce it.
 * ---------------------------------------------------------------------------------------- */
static void flood_frame(const void *vctx, long f, Work *w) {
    const Ctx *c = (const Ctx *)vctx;
    const int E = c->E, N = c->N, M = c->M;
    const double *L = c->llr + (size_t)f * N;
    double *v2c = w->a, *c2v = w->b, *tot = w->tot, *th = w->th;
    uint8_t *d = w->d;
    for (int e = 0; e < E; ++e) { v2c[e] = L[c->col_idx[e]]; c2v[e] = 0.0; }
    int l, ok = 0;
    for (l = 1;; ++l) {
        for (int m = 0; m < M; ++m) {
            int b = c->row_ptr[m], dd = c->row_ptr[m + 1] - b;
            for (int k = 0; k < dd; ++k) th[k] = tanh(0.5 * clip(v2c[b + k], c->llr_max));
            for (int k = 0; k < dd; ++k) {
                double p = 1.0;
                for (int j = 0; j < dd; ++j)
                    if (j != k) p *= th[j];
                if (p > 1.0 - 1e-15) p = 1.0 - 1e-15;
                if (p < -(1.0 - 1e-15)) p = -(1.0 - 1e-15);
                c2v[b + k] = clip(log((1.0 + p) / (1.0 - p)), c->llr_max);
            }
        }
        for (int n = 0; n < N; ++n) {
            double s = L[n];
            for (int i = c->col_ptr[n]; i < c->col_ptr[n + 1]; ++i) s += c2v[c->col_edge[i]];
            tot[n] = s;
            for (int i = c->col_ptr[n]; i < c->col_ptr[n + 1]; ++i) v2c[c->col_edge[i]] = s - c2v[c->col_edge[i]];
            d[n] = s < 0.0;
        }
        ok = 1;
        for (int m = 0; m < M && ok; ++m) {
            int p = 0;
            for (int e = c->row_ptr[m]; e < c->row_ptr[m + 1]; ++e) p ^= d[c->col_idx[e]];
            if (p) ok = 0;
        }
        if ((ok && c->early_stop) || l >= c->max_iter) break;
    }
    write_outputs(c, f, l, ok, tot, d, c2v);
}

/* ------------------------------------------------------------------------------------------
 * Textbook row-serial layered BP in posterior form: rows in index order; for each row, the
 * extrinsic inputs are t = P_n - R_{m,n}, the row's new messages R follow the tanh rule, and
 * P_n = t + R_{m,n}.  The NDGSBP schedule with one CN per group, r = 0 and the groups in row
 * order must reproduce it.
 * ---------------------------------------------------------------------------------------- */
static void layered_frame(const void *vctx, long f, Work *w) {
    const Ctx *c = (const Ctx *)vctx;
    const int E = c->E, N = c->N, M = c->M;
    const double *L = c->llr + (size_t)f * N;
    double *R = w->a, *t = w->b, *P = w->tot, *th = w->th;
    uint8_t *d = w->d;
    for (int e = 0; e < E; ++e) R[e] = 0.0;
    for (int n = 0; n < N; ++n) P[n] = L[n];
    int l, ok = 0;
    for (l = 1;; ++l) {
        for (int m = 0; m < M; ++m) {
            int b = c->row_ptr[m], dd = c->row_ptr[m + 1] - b;
            for (int k = 0; k < dd; ++k) {
                t[b + k] = P[c->col_idx[b + k]] - R[b + k];
                th[k] = tanh(0.5 * clip(t[b + k], c->llr_max));
            }
            for (int k = 0; k < dd; ++k) {
                double p = 1.0;
                for (int j = 0; j < dd; ++j)
                    if (j != k) p *= th[j];
                if (p > 1.0 - 1e-15) p = 1.0 - 1e-15;
                if (p < -(1.0 - 1e-15)) p = -(1.0 - 1e-15);
                R[b + k] = clip(2.0 * atanh(p), c->llr_max);
                P[c->col_idx[b + k]] = t[b + k] + R[b + k];
            }
        }
        for (int n = 0; n < N; ++n) d[n] = P[n] < 0.0;
        ok = 1;
        for (int m = 0; m < M && ok; ++m) {
            int p = 0;
            for (int e = c->row_ptr[m]; e < c->row_ptr[m + 1]; ++e) p ^= d[c->col_idx[e]];
            if (p) ok = 0;
        }
        if ((ok && c->early_stop) || l >= c->max_iter) break;
    }
    write_outputs(c, f, l, ok, P, d, R);
}

/* ------------------------------------------------------------------------------------------
 * Textbook horizontal group-shuffled BP in posterior form, for any list of CN groups: for each
 * group, every edge of its CNs first takes t = P_n - R_{m,n} from the posteriors as they stood
 * at the start of the group, then each CN's new messages follow the tanh rule, then
 * P_n += R_new - R_old over the group's edges.  A second, independent formulation of the
 * schedule that oracle_ndgsbp_decode writes with explicit VN->CN messages.
 * ---------------------------------------------------------------------------------------- */
static void group_posterior_frame(const void *vctx, long f, Work *w) {
    const Ctx *c = (const Ctx *)vctx;
    const int E = c->E, N = c->N, M = c->M;
    const double *L = c->llr + (size_t)f * N;
    double *R = w->a, *t = w->b, *P = w->tot, *th = w->th;
    uint8_t *d = w->d;
    for (int e = 0; e < E; ++e) R[e] = 0.0;
    for (int n = 0; n < N; ++n) P[n] = L[n];
    int l, ok = 0;
    for (l = 1;; ++l) {
        for (int g = 0; g < c->G; ++g) {
            for (int i = c->grp_ptr[g]; i < c->grp_ptr[g + 1]; ++i) {
                int m = c->grp_cn[i];
                for (int e = c->row_ptr[m]; e < c->row_ptr[m + 1]; ++e) t[e] = P[c->col_idx[e]] - R[e];
            }
            for (int i = c->grp_ptr[g]; i < c->grp_ptr[g + 1]; ++i) {
                int m = c->grp_cn[i];
                int b = c->row_ptr[m], dd = c->row_ptr[m + 1] - b;
                for (int k = 0; k < dd; ++k) th[k] = tanh(0.5 * clip(t[b + k], c->llr_max));
                for (int k = 0; k < dd; ++k) {
                    double p = 1.0;
                    for (int j = 0; j < dd; ++j)
                        if (j != k) p *= th[j];
                    if (p > 1.0 - 1e-15) p = 1.0 - 1e-15;
                    if (p < -(1.0 - 1e-15)) p = -(1.0 - 1e-15);
                    double rn = clip(2.0 * atanh(p), c->llr_max);
                    P[c->col_idx[b + k]] += rn - R[b + k];
                    R[b + k] = rn;
                }
            }
        }
        for (int n = 0; n < N; ++n) d[n] = P[n] < 0.0;
        ok = 1;
        for (int m = 0; m < M && ok; ++m) {
            int p = 0;
            for (int e = c->row_ptr[m]; e < c->row_ptr[m + 1]; ++e) p ^= d[c->col_idx[e]];
            if (p) ok = 0;
        }
        if ((ok && c->early_stop) || l >= c->max_iter) break;
    }
    write_outputs(c, f, l, ok, P, d, R);
}

/* ------------------------------------------------------------------------------------------
 * Frame-parallel driver: one frame per task, each frame computed by one thread.
 * ---------------------------------------------------------------------------------------- */
static void *worker(void *arg) {
    Ctx *c = (Ctx *)arg;
    Work w;
    size_t E = (size_t)(c->E > 0 ? c->E : 1), N = (size_t)c->N;
    w.a = (double *)malloc(sizeof(double) * E);
    w.b = (double *)malloc(sizeof(double) * E);
    w.tot = (double *)malloc(sizeof(double) * N);
    w.th = (double *)malloc(sizeof(double) * (size_t)(c->max_deg_row + 1));
    w.d = (uint8_t *)malloc(N);
    w.mark = (uint8_t *)malloc(N);
    w.touched = (int *)malloc(sizeof(int) * N);
    void *ret = NULL;
    if (!w.a || !w.b || !w.tot || !w.th || !w.d || !w.mark || !w.touched) {
        ret = (void *)1;
    } else {
        for (;;) {
            pthread_mutex_lock(&c->lock);
            long f = c->next_frame++;
            pthread_mutex_unlock(&c->lock);
            if (f >= c->n_frames) break;
            c->frame_fn(c, f, &w);
        }
    }
    free(w.a); free(w.b); free(w.tot); free(w.th); free(w.d); free(w.mark); free(w.touched);
    return ret;
}

static int run_frames(Ctx *c, int n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    c->next_frame = 0;
    pthread_mutex_init(&c->lock, NULL);
    pthread_t th[256];
    int started = 0, rc = ORACLE_OK;
    for (int i = 1; i < n_threads; ++i)
        if (pthread_create(&th[started], NULL, worker, c) == 0) started++;
    if (worker(c) != NULL) rc = ORACLE_ENOMEM;
    for (int i = 0; i < started; ++i) {
        void *ret = NULL;
        pthread_join(th[i], &ret);
        if (ret) rc = ORACLE_ENOMEM;
    }
    pthread_mutex_destroy(&c->lock);
    return rc;
}

static int setup(Ctx *c, int M, int N, const int *row_ptr, const int *col_idx, const double *llr,
                 long n_frames, int max_iter, double llr_max, int early_stop, uint8_t *hard,
                 int *iters, uint8_t *synd_ok, double *total, double *c2v_out) {
    memset(c, 0, sizeof(*c));
    if (M < 1 || N < 1 || n_frames < 0 || max_iter < 1) return ORACLE_EINVAL;
    c->M = M; c->N = N; c->E = row_ptr[M];
    c->row_ptr = row_ptr; c->col_idx = col_idx;
    c->llr = llr; c->n_frames = n_frames; c->max_iter = max_iter; c->llr_max = llr_max;
    c->early_stop = early_stop; c->hard = hard; c->iters = iters; c->synd_ok = synd_ok;
    c->total = total; c->c2v_out = c2v_out;
    c->stop_after_subiters = -1;
    c->n_groupings = 1;
    return build_columns(c);
}

static void teardown(Ctx *c) {
    free(c->col_ptr);
    free(c->col_edge);
    free(c->edge_row);
}

/* NDGSBP decoder.  grp_ptr has n_groupings * (G + 1) entries (grouping k's pointers at
 * k * (G + 1)) into the shared grp_cn array; with n_groupings > 1 the groups are redrawn per
 * iteration by cycling through the given groupings.  stop_after_subiters > 0 stops after that
 * many sub-iterations (group updates) and reports the state there.  Outputs per frame: hard
 * decisions [N] (uint8), iterations, syndrome flag, optional total LLR [N] and optional CN->VN
 * messages [E] in CSR edge order. */
int oracle_ndgsbp_decode(int M, int N, const int *row_ptr, const int *col_idx, int G,
                         const int *grp_ptr, const int *grp_cn, int n_groupings, const double *llr,
                         long n_frames, int max_iter, double llr_max, int early_stop,
                         int stop_after_subiters, uint8_t *hard, int *iters, uint8_t *synd_ok,
                         double *total, double *c2v_out, int n_threads) {
    Ctx c;
    int rc = setup(&c, M, N, row_ptr, col_idx, llr, n_frames, max_iter, llr_max, early_stop, hard,
                   iters, synd_ok, total, c2v_out);
    if (rc) { teardown(&c); return rc; }
    if (G < 1 || n_groupings < 1) { teardown(&c); return ORACLE_EINVAL; }
    for (int k = 0; k < n_groupings; ++k) {
        const int *gp = grp_ptr + (size_t)k * (G + 1);
        for (int g = 0; g < G; ++g)
            for (int i = gp[g]; i < gp[g + 1]; ++i)
                if (grp_cn[i] < 0 || grp_cn[i] >= M) { teardown(&c); return ORACLE_EINVAL; }
    }
    c.G = G; c.grp_ptr = grp_ptr; c.grp_cn = grp_cn; c.n_groupings = n_groupings;
    c.stop_after_subiters = stop_after_subiters;
    c.frame_fn = ndgsbp_frame;
    rc = run_frames(&c, n_threads);
    teardown(&c);
    return rc;
}

int oracle_group_posterior_decode(int M, int N, const int *row_ptr, const int *col_idx, int G,
                                  const int *grp_ptr, const int *grp_cn, const double *llr,
                                  long n_frames, int max_iter, double llr_max, int early_stop,
                                  uint8_t *hard, int *iters, uint8_t *synd_ok, double *total,
                                  double *c2v_out, int n_threads) {
    Ctx c;
    int rc = setup(&c, M, N, row_ptr, col_idx, llr, n_frames, max_iter, llr_max, early_stop, hard,
                   iters, synd_ok, total, c2v_out);
    if (rc) { teardown(&c); return rc; }
    if (G < 1) { teardown(&c); return ORACLE_EINVAL; }
    for (int i = 0; i < grp_ptr[G]; ++i)
        if (grp_cn[i] < 0 || grp_cn[i] >= M) { teardown(&c); return ORACLE_EINVAL; }
    c.G = G; c.grp_ptr = grp_ptr; c.grp_cn = grp_cn;
    c.frame_fn = group_posterior_frame;
    rc = run_frames(&c, n_threads);
    teardown(&c);
    return rc;
}

int oracle_flood_decode(int M, int N, const int *row_ptr, const int *col_idx, const double *llr,
                        long n_frames, int max_iter, double llr_max, int early_stop, uint8_t *hard,
                        int *iters, uint8_t *synd_ok, double *total, double *c2v_out, int n_threads) {
    Ctx c;
    int rc = setup(&c, M, N, row_ptr, col_idx, llr, n_frames, max_iter, llr_max, early_stop, hard,
                   iters, synd_ok, total, c2v_out);
    if (rc) { teardown(&c); return rc; }
    c.frame_fn = flood_frame;
    rc = run_frames(&c, n_threads);
    teardown(&c);
    return rc;
}

int oracle_layered_decode(int M, int N, const int *row_ptr, const int *col_idx, const double *llr,
                          long n_frames, int max_iter, double llr_max, int early_stop, uint8_t *hard,
                          int *iters, uint8_t *synd_ok, double *total, double *c2v_out, int n_threads) {
    Ctx c;
    int rc = setup(&c, M, N, row_ptr, col_idx, llr, n_frames, max_iter, llr_max, early_stop, hard,
                   iters, synd_ok, total, c2v_out);
    if (rc) { teardown(&c); return rc; }
    c.frame_fn = layered_frame;
    rc = run_frames(&c, n_threads);
    teardown(&c);
    return rc;
}

/* ------------------------------------------------------------------------------------------
 * Vertical group shuffled BP, the VN-partitioned serial schedule of Sec. I: the VNs are split
 * into G groups that are processed one after another within an iteration.  In sub-iteration g
 * every VN n of group g receives from each of its CNs m the message of Eq. (1), computed from the
 * VN->CN messages of m's other VNs as they stand at the start of the sub-iteration (VNs of
 * earlier groups already updated in this iteration, the others not yet); only then do the VNs
 * of the group send their new messages, L_{n->m} = L_n + sum over the other CNs m' of n of
 * L_{m'->n} (Eq. (2)).  With one group this is flooding.  After the last group: Eq. (3), the
 * decision and the syndrome of Step 4.
 * ---------------------------------------------------------------------------------------- */
static void vertical_frame(const void *vctx, long f, Work *w) {
    const Ctx *c = (const Ctx *)vctx;
    const int E = c->E, N = c->N;
    const double *L = c->llr + (size_t)f * N;
    double *v2c = w->a, *c2v = w->b, *tot = w->tot, *th = w->th;
    uint8_t *d = w->d;
    for (int e = 0; e < E; ++e) { v2c[e] = L[c->col_idx[e]]; c2v[e] = 0.0; }
    int l, ok = 0;
    for (l = 1;; ++l) {
        for (int g = 0; g < c->G; ++g) {
            /* CN->VN messages into the group's VNs (Eq. (1)), from the current VN->CN messages */
            for (int i = c->grp_ptr[g]; i < c->grp_ptr[g + 1]; ++i) {
                const int n = c->grp_cn[i];
                for (int a = c->col_ptr[n]; a < c->col_ptr[n + 1]; ++a) {
                    const int e = c->col_edge[a], m = c->edge_row[e];
                    const int b = c->row_ptr[m], dd = c->row_ptr[m + 1] - b;
                    double prod = 1.0;
                    for (int j = 0; j < dd; ++j) {
                        th[j] = tanh(0.5 * clip(v2c[b + j], c->llr_max));
                        if (b + j != e) prod *= th[j];
                    }
                    const double lim = 1.0 - 1e-15;
                    if (prod > lim) prod = lim;
                    if (prod < -lim) prod = -lim;
                    c2v[e] = clip(2.0 * atanh(prod), c->llr_max);
                }
            }
            /* then the group's VN->CN messages (Eq. (2), a direct sum over the other CNs) */
            for (int i = c->grp_ptr[g]; i < c->grp_ptr[g + 1]; ++i) {
                const int n = c->grp_cn[i];
                for (int a = c->col_ptr[n]; a < c->col_ptr[n + 1]; ++a) {
                    double s = L[n];
                    for (int a2 = c->col_ptr[n]; a2 < c->col_ptr[n + 1]; ++a2)
                        if (a2 != a) s += c2v[c->col_edge[a2]];
                    v2c[c->col_edge[a]] = s;
                }
            }
        }
        ok = total_and_syndrome(c, L, c2v, tot, d);
        if ((ok && c->early_stop) || l >= c->max_iter) break;
    }
    write_outputs(c, f, l, ok, tot, d, c2v);
}

/* Vertical group shuffled decoder: grp_ptr[G + 1] into grp_vn, a partition of the N VNs (each
 * exactly once).  Outputs as oracle_ndgsbp_decode. */
int oracle_vertical_decode(int M, int N, const int *row_ptr, const int *col_idx, int G, const int *grp_ptr,
                           const int *grp_vn, const double *llr, long n_frames, int max_iter, double llr_max,
                           int early_stop, uint8_t *hard, int *iters, uint8_t *synd_ok, double *total,
                           double *c2v_out, int n_threads) {
    Ctx c;
    int rc = setup(&c, M, N, row_ptr, col_idx, llr, n_frames, max_iter, llr_max, early_stop, hard,
                   iters, synd_ok, total, c2v_out);
    if (rc) { teardown(&c); return rc; }
    if (G < 1 || grp_ptr[0] != 0 || grp_ptr[G] != N) { teardown(&c); return ORACLE_EINVAL; }
    uint8_t *seen = (uint8_t *)calloc((size_t)N, 1);
    c.edge_row = (int *)malloc(sizeof(int) * (size_t)(c.E > 0 ? c.E : 1));
    if (!seen || !c.edge_row) { free(seen); teardown(&c); return ORACLE_ENOMEM; }
    for (int i = 0; i < N; ++i) {
        if (grp_vn[i] < 0 || grp_vn[i] >= N || seen[grp_vn[i]]) { free(seen); teardown(&c); return ORACLE_EINVAL; }
        seen[grp_vn[i]] = 1;
    }
    free(seen);
    for (int g = 0; g < G; ++g)
        if (grp_ptr[g + 1] < grp_ptr[g]) { teardown(&c); return ORACLE_EINVAL; }
    for (int m = 0; m < M; ++m)
        for (int e = row_ptr[m]; e < row_ptr[m + 1]; ++e) c.edge_row[e] = m;
    c.G = G; c.grp_ptr = grp_ptr; c.grp_cn = grp_vn;
    c.frame_fn = vertical_frame;
    rc = run_frames(&c, n_threads);
    teardown(&c);
    return rc;
}

/* ------------------------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11).  One round maps counter (c0, c1, c2, c3) under key (k0, k1) to
 *   (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
 * with the 64-bit products of the multipliers M0, M1; the key grows by the Weyl increments
 * (W0, W1) between rounds.  Ten rounds.
 * ---------------------------------------------------------------------------------------- */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* BPSK/AWGN channel LLRs (Sec. II-C: L_n = 2 y_n / sigma^2, y_n = (1 - 2 c_n) + sigma z_n) with
 * sigma^2 = 1 / (2 R 10^(EbN0/10)).  The normal samples follow one fixed definition that the
 * CUDA generator implements on its own:
 *   key = (seed mod 2^32, seed div 2^32); for frame f and block b, counter = (b, f mod 2^32,
 *   f div 2^32, 0); the four outputs x_i give u_i = ((x_i >> 9) + 1/2) 2^-23 in (0, 1) (a value
 *   every binary32 implementation represents exactly);
 *   Box-Muller: z_{4b}   = sqrt(-2 ln u_0) cos(2 pi u_1),  z_{4b+1} = sqrt(-2 ln u_0) sin(2 pi u_1),
 *               z_{4b+2} = sqrt(-2 ln u_2) cos(2 pi u_3),  z_{4b+3} = sqrt(-2 ln u_2) sin(2 pi u_3).
 * codeword: NULL (all-zero word) or [N] bits. */
int oracle_awgn_llr(int N, long n_frames, double ebn0_db, double rate, uint64_t seed,
                    const uint8_t *codeword, double *llr) {
    if (N < 1 || n_frames < 0 || !(rate > 0.0)) return ORACLE_EINVAL;
    const double sigma2 = 1.0 / (2.0 * rate * pow(10.0, ebn0_db / 10.0));
    const double sigma = sqrt(sigma2);
    const double two_pi = 6.283185307179586476925286766559;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (long f = 0; f < n_frames; ++f) {
        for (int b = 0; 4 * b < N; ++b) {
            uint32_t ctr[4] = {(uint32_t)b, (uint32_t)((uint64_t)f), (uint32_t)((uint64_t)f >> 32), 0u};
            uint32_t x[4];
            oracle_philox4x32_10(ctr, key, x);
            double u[4], z[4];
            for (int i = 0; i < 4; ++i) u[i] = ((double)(x[i] >> 9) + 0.5) * (1.0 / 8388608.0);
            double r0 = sqrt(-2.0 * log(u[0])), r1 = sqrt(-2.0 * log(u[2]));
            z[0] = r0 * cos(two_pi * u[1]);
            z[1] = r0 * sin(two_pi * u[1]);
            z[2] = r1 * cos(two_pi * u[3]);
            z[3] = r1 * sin(two_pi * u[3]);
            for (int i = 0; i < 4; ++i) {
                int n = 4 * b + i;
                if (n >= N) break;
                double xmod = (codeword && codeword[n]) ? -1.0 : 1.0;
                double y = xmod + sigma * z[i];
                llr[(size_t)f * N + n] = 2.0 * y / sigma2;
            }
        }
    }
    return ORACLE_OK;
}
