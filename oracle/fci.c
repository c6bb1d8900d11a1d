/*
 * ORACLE -- test infrastructure only.  Nothing in the product path may link,
 * load or call this file; only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py use it.
 *
 * Plain determinant-basis action of the ab-initio Hamiltonian (Eq. 1, Sec. 2.1;
 * full-CI expansion Eq. fulltensor) in the chemist convention
 *     H = sum_ij t_ij sum_s a+_is a_js
 *       + 1/2 sum_ijkl (ij|kl) sum_st a+_is a+_kt a_lt a_js ,
 * evaluated term by term on Slater determinants with no factorisation.
 *
 * Spin-orbitals are ordered p = 2*i + s (s = 0 alpha, s = 1 beta); a determinant
 * is the product of creators with ascending p on the vacuum.  The basis of the
 * (na, nb) space is alpha-string x beta-string, each string ranked among the
 * masks with that popcount in ascending integer order: index = ra * nbeta + rb.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int L, na, nb;
    long nA, nB;
    uint32_t *amask, *bmask;   /* strings in rank order */
    int32_t *arank, *brank;    /* mask -> rank (or -1), size 2^L */
} space_t;

static int popc(uint32_t x) { return __builtin_popcount(x); }

static long enumerate(int L, int n, uint32_t *out, int32_t *rank) {
    long c = 0;
    for (uint32_t m = 0; m < (1u << L); ++m) {
        if (popc(m) == n) {
            if (out) out[c] = m;
            if (rank) rank[m] = (int32_t)c;
            ++c;
        } else if (rank) {
            rank[m] = -1;
        }
    }
    return c;
}

static int space_init(space_t *sp, int L, int na, int nb) {
    if (L < 1 || L > 24 || na < 0 || nb < 0 || na > L || nb > L) return -1;
    sp->L = L; sp->na = na; sp->nb = nb;
    sp->nA = enumerate(L, na, NULL, NULL);
    sp->nB = enumerate(L, nb, NULL, NULL);
    sp->amask = (uint32_t *)malloc(sizeof(uint32_t) * sp->nA);
    sp->bmask = (uint32_t *)malloc(sizeof(uint32_t) * sp->nB);
    sp->arank = (int32_t *)malloc(sizeof(int32_t) * (1u << L));
    sp->brank = (int32_t *)malloc(sizeof(int32_t) * (1u << L));
    enumerate(L, na, sp->amask, sp->arank);
    enumerate(L, nb, sp->bmask, sp->brank);
    return 0;
}

static void space_free(space_t *sp) {
    free(sp->amask); free(sp->bmask); free(sp->arank); free(sp->brank);
}

/* A determinant during operator application: alpha and beta occupation masks. */
typedef struct { uint32_t a, b; int ok; double sign; } det_t;

/* number of occupied spin-orbitals with index below p = 2i+s */
static int below(const det_t *d, int i, int s) {
    uint32_t low = (i == 0) ? 0u : ((1u << i) - 1u);
    int c = popc(d->a & low) + popc(d->b & low);
    if (s == 1) c += (d->a >> i) & 1u;
    return c;
}

static void annihilate(det_t *d, int i, int s) {
    if (!d->ok) return;
    uint32_t *m = s ? &d->b : &d->a;
    if (!((*m >> i) & 1u)) { d->ok = 0; return; }
    if (below(d, i, s) & 1) d->sign = -d->sign;
    *m &= ~(1u << i);
}

static void create(det_t *d, int i, int s) {
    if (!d->ok) return;
    uint32_t *m = s ? &d->b : &d->a;
    if ((*m >> i) & 1u) { d->ok = 0; return; }
    if (below(d, i, s) & 1) d->sign = -d->sign;
    *m |= (1u << i);
}

/*
 * y = H x on the (na, nb) determinant space.  Gather form: for every output
 * determinant D, H|D> is expanded term by term and y[D] += <D'|H|D> x[D'];
 * H is real symmetric so <D'|H|D> = <D|H|D'>.
 */
int oracle_fci_sigma(int L, int na, int nb, const double *t, const double *v,
                     const double *x, double *y) {
    space_t sp;
    if (space_init(&sp, L, na, nb)) return -1;
    const long nB = sp.nB;
    const long n = sp.nA * sp.nB;
    const long L2 = (long)L * L, L3 = L2 * L;
#pragma omp parallel for schedule(dynamic, 64)
    for (long D = 0; D < n; ++D) {
        det_t d0 = { sp.amask[D / nB], sp.bmask[D % nB], 1, 1.0 };
        double acc = 0.0;
        /* one-body part */
        for (int s = 0; s < 2; ++s)
            for (int j = 0; j < L; ++j) {
                det_t d1 = d0; annihilate(&d1, j, s);
                if (!d1.ok) continue;
                for (int i = 0; i < L; ++i) {
                    double tij = t[(long)i * L + j];
                    if (tij == 0.0) continue;
                    det_t d2 = d1; create(&d2, i, s);
                    if (!d2.ok) continue;
                    long Dp = (long)sp.arank[d2.a] * nB + sp.brank[d2.b];
                    acc += tij * d2.sign * x[Dp];
                }
            }
        /* two-body part: 1/2 (ij|kl) a+_is a+_kt a_lt a_js, applied right to left */
        for (int s = 0; s < 2; ++s)
            for (int j = 0; j < L; ++j) {
                det_t d1 = d0; annihilate(&d1, j, s);
                if (!d1.ok) continue;
                for (int tt = 0; tt < 2; ++tt)
                    for (int l = 0; l < L; ++l) {
                        det_t d2 = d1; annihilate(&d2, l, tt);
                        if (!d2.ok) continue;
                        for (int k = 0; k < L; ++k) {
                            det_t d3 = d2; create(&d3, k, tt);
                            if (!d3.ok) continue;
                            for (int i = 0; i < L; ++i) {
                                double g = v[(long)i * L3 + (long)j * L2 + (long)k * L + l];
                                if (g == 0.0) continue;
                                det_t d4 = d3; create(&d4, i, s);
                                if (!d4.ok) continue;
                                long Dp = (long)sp.arank[d4.a] * nB + sp.brank[d4.b];
                                acc += 0.5 * g * d4.sign * x[Dp];
                            }
                        }
                    }
            }
        y[D] = acc;
    }
    space_free(&sp);
    return 0;
}

/*
 * Expectation values needed for the reduced density matrices:
 *   g1[i*L+j]            = <x| sum_s a+_is a_js |y>
 *   g2[((i*L+j)*L+k)*L+l] = <x| sum_st a+_is a+_kt a_lt a_js |y>
 * (Gamma_ijkl in the chemist ordering, so that E = sum t g1 + 1/2 sum v g2).
 */
int oracle_fci_rdm12(int L, int na, int nb, const double *x, const double *y,
                     double *g1, double *g2) {
    space_t sp;
    if (space_init(&sp, L, na, nb)) return -1;
    const long nB = sp.nB;
    const long n = sp.nA * sp.nB;
    const long L2 = (long)L * L, L3 = L2 * L, L4 = L3 * L;
    memset(g1, 0, sizeof(double) * L2);
    memset(g2, 0, sizeof(double) * L4);
#pragma omp parallel
    {
        double *p1 = (double *)calloc(L2, sizeof(double));
        double *p2 = (double *)calloc(L4, sizeof(double));
#pragma omp for schedule(dynamic, 64)
        for (long D = 0; D < n; ++D) {
            double yD = y[D];
            if (yD == 0.0) continue;
            det_t d0 = { sp.amask[D / nB], sp.bmask[D % nB], 1, 1.0 };
            for (int s = 0; s < 2; ++s)
                for (int j = 0; j < L; ++j) {
                    det_t d1 = d0; annihilate(&d1, j, s);
                    if (!d1.ok) continue;
                    for (int i = 0; i < L; ++i) {
                        det_t d2 = d1; create(&d2, i, s);
                        if (!d2.ok) continue;
                        long Dp = (long)sp.arank[d2.a] * nB + sp.brank[d2.b];
                        p1[(long)i * L + j] += x[Dp] * d2.sign * yD;
                    }
                    for (int tt = 0; tt < 2; ++tt)
                        for (int l = 0; l < L; ++l) {
                            det_t d2 = d1; annihilate(&d2, l, tt);
                            if (!d2.ok) continue;
                            for (int k = 0; k < L; ++k) {
                                det_t d3 = d2; create(&d3, k, tt);
                                if (!d3.ok) continue;
                                for (int i = 0; i < L; ++i) {
                                    det_t d4 = d3; create(&d4, i, s);
                                    if (!d4.ok) continue;
                                    long Dp = (long)sp.arank[d4.a] * nB + sp.brank[d4.b];
                                    p2[(long)i * L3 + (long)j * L2 + (long)k * L + l] += x[Dp] * d4.sign * yD;
                                }
                            }
                        }
                }
        }
#pragma omp critical
        {
            for (long q = 0; q < L2; ++q) g1[q] += p1[q];
            for (long q = 0; q < L4; ++q) g2[q] += p2[q];
        }
        free(p1); free(p2);
    }
    space_free(&sp);
    return 0;
}

/* alpha / beta string tables in rank order (for the basis maps of the harness) */
long oracle_fci_strings(int L, int n, uint32_t *out) {
    if (L < 1 || L > 24) return -1;
    return enumerate(L, n, out, NULL);
}
