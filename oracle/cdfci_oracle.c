/*
 * CPU oracle for the CDFCI / mCDFCI column update.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file's library.  It shares
 * no code, header, table or constant with the CUDA library; the product path
 * never calls it.
 *
 * Everything here is plain, serial and written for a reader checking it
 * against the paper by eye:
 *
 *   - Section "Hamiltonian Representations", Eq. (general-ham):
 *       H = sum_{PQ} h_PQ a+_P a_Q + 1/2 sum_{PQRS} v_PQRS a+_P a+_Q a_S a_R
 *     over spin-orbitals P = (p, sigma).  Real spatial integrals are given as
 *     h[p][q] and chemists' g[p][q][r][s] = (pq|rs); the physicists' element
 *     of Eq. (2int) is v_{PQRS} = (pr|qs) delta(sP,sR) delta(sQ,sS).
 *   - H_IJ = <Phi_I|H|Phi_J> is evaluated by LITERALLY applying every term of
 *     the operator to the occupation bitstring of Phi_J (column_literal).  This
 *     is the definition layer.
 *   - Eq. (entry) (Slater-Condon rules) is restated in spin-orbital form in
 *     column_sc; it is checked against column_literal by the tests.
 *   - Algorithm 1 (CDFCI) and Algorithm 2 (mCDFCI) are followed step by step
 *     in orc_step, with the scalars c^T c and c^T H c kept in binary128 as the
 *     section on the WaveFunction class prescribes.
 *   - The step size follows the appendix "Determining Step Size": Cardano's
 *     method on the cubic derivative of the quartic, then Newton refinement.
 *
 * Conventions (readings of points the paper leaves open):
 *   - Jordan-Wigner order is alpha-block first: spin-orbital (p, alpha) has
 *     index p, (p, beta) has index N + p.  A determinant is the pair of 64-bit
 *     words (A, B): bit p of A is (p, alpha), bit p of B is (p, beta).
 *   - a_Q on |n> gives (-1)^(number of occupied spin-orbitals with index < Q)
 *     times |n with Q cleared>, or 0 if Q is empty; a+_P likewise.
 *   - A column entry exists iff its value is a nonzero double.
 *   - Ties in |gradient| go to the smaller key, compared as the unsigned
 *     128-bit number (B << 64) | A.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#if defined(__x86_64__) || defined(__i386__)
typedef __float128 quad;          /* IEEE binary128 (software) */
#else
typedef long double quad;         /* binary128 on aarch64 Linux */
#endif

/* ------------------------------------------------------------------------ */
/* Determinants and ladder operators                                         */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t a, b; } det_t;

static int popc(uint64_t x) { return __builtin_popcountll(x); }

static uint64_t below(int bit) { return bit <= 0 ? 0ULL : (bit >= 64 ? ~0ULL : ((1ULL << bit) - 1ULL)); }

/* occupation of spin-orbital P in determinant d (N spatial orbitals) */
static int occupied(const det_t *d, int N, int P) {
    if (P < N) return (int)((d->a >> P) & 1ULL);
    return (int)((d->b >> (P - N)) & 1ULL);
}

/* number of occupied spin-orbitals with Jordan-Wigner index < P */
static int occupied_below(const det_t *d, int N, int P) {
    if (P < N) return popc(d->a & below(P));
    return popc(d->a) + popc(d->b & below(P - N));
}

static void flip(det_t *d, int N, int P) {
    if (P < N) d->a ^= (1ULL << P);
    else d->b ^= (1ULL << (P - N));
}

/* a_P applied in place: returns the sign (+1/-1), or 0 if the state vanishes */
static int annihilate(det_t *d, int N, int P) {
    if (!occupied(d, N, P)) return 0;
    int s = (occupied_below(d, N, P) & 1) ? -1 : 1;
    flip(d, N, P);
    return s;
}

/* a+_P applied in place: returns the sign, or 0 if the state vanishes */
static int create(det_t *d, int N, int P) {
    if (occupied(d, N, P)) return 0;
    int s = (occupied_below(d, N, P) & 1) ? -1 : 1;
    flip(d, N, P);
    return s;
}

/* spin-orbital one-body integral h_PQ = h_pq delta(sP, sQ) */
static double h_so(int N, const double *h, int P, int Q) {
    if ((P < N) != (Q < N)) return 0.0;
    return h[(P % N) * N + (Q % N)];
}

/* physicists' spin-orbital integral v_PQRS = (pr|qs) delta(sP,sR) delta(sQ,sS), Eq. (2int) */
static double v_so(int N, const double *g, int P, int Q, int R, int S) {
    if ((P < N) != (R < N)) return 0.0;
    if ((Q < N) != (S < N)) return 0.0;
    int p = P % N, q = Q % N, r = R % N, s = S % N;
    return g[(((size_t)p * N + r) * N + q) * N + s];
}

static int det_less(det_t x, det_t y) {   /* unsigned 128-bit (b << 64) | a */
    if (x.b != y.b) return x.b < y.b;
    return x.a < y.a;
}

/* ------------------------------------------------------------------------ */
/* A plain open-addressing map det -> index (linear probing)                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t cap;          /* power of two */
    int64_t n;
    det_t *key;
    int64_t *val;         /* index payload, -1 = empty */
} dmap;

static uint64_t det_hash(det_t d) {
    /* any deterministic mixing is fine for the oracle's own map */
    uint64_t x = d.a * 0x9E3779B97F4A7C15ULL ^ (d.b + 0x632BE59BD9B4E019ULL + (d.a << 7));
    x ^= x >> 31; x *= 0xD6E8FEB86659FD93ULL; x ^= x >> 32;
    return x;
}

static int dmap_init(dmap *m, int64_t cap_hint) {
    int64_t cap = 16;
    while (cap < 2 * cap_hint) cap <<= 1;
    m->cap = cap; m->n = 0;
    m->key = (det_t *)calloc((size_t)cap, sizeof(det_t));
    m->val = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    if (!m->key || !m->val) return -1;
    for (int64_t i = 0; i < cap; i++) m->val[i] = -1;
    return 0;
}

static void dmap_free(dmap *m) { free(m->key); free(m->val); m->key = 0; m->val = 0; }

static int dmap_grow(dmap *m);

/* returns stored index, or -1 if absent */
static int64_t dmap_get(const dmap *m, det_t d) {
    uint64_t mask = (uint64_t)m->cap - 1;
    for (uint64_t p = det_hash(d) & mask;; p = (p + 1) & mask) {
        if (m->val[p] < 0) return -1;
        if (m->key[p].a == d.a && m->key[p].b == d.b) return m->val[p];
    }
}

/* inserts d with payload v if absent; returns the stored payload */
static int64_t dmap_put(dmap *m, det_t d, int64_t v) {
    if (2 * (m->n + 1) > m->cap) { if (dmap_grow(m)) return -2; }
    uint64_t mask = (uint64_t)m->cap - 1;
    for (uint64_t p = det_hash(d) & mask;; p = (p + 1) & mask) {
        if (m->val[p] < 0) { m->key[p] = d; m->val[p] = v; m->n++; return v; }
        if (m->key[p].a == d.a && m->key[p].b == d.b) return m->val[p];
    }
}

static int dmap_grow(dmap *m) {
    dmap bigger;
    if (dmap_init(&bigger, m->cap)) return -1;
    for (int64_t i = 0; i < m->cap; i++)
        if (m->val[i] >= 0) dmap_put(&bigger, m->key[i], m->val[i]);
    dmap_free(m);
    *m = bigger;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Columns of H                                                              */
/* ------------------------------------------------------------------------ */

/* growable list of (det, value) */
typedef struct { int64_t n, cap; det_t *d; double *v; dmap idx; } colbuf;

static int colbuf_init(colbuf *c, int64_t hint) {
    c->n = 0; c->cap = hint > 16 ? hint : 16;
    c->d = (det_t *)malloc((size_t)c->cap * sizeof(det_t));
    c->v = (double *)malloc((size_t)c->cap * sizeof(double));
    if (!c->d || !c->v) return -1;
    return dmap_init(&c->idx, hint);
}
static void colbuf_free(colbuf *c) { free(c->d); free(c->v); dmap_free(&c->idx); }

/* accumulate value x onto the entry for determinant d */
static int colbuf_add(colbuf *c, det_t d, double x) {
    int64_t k = dmap_get(&c->idx, d);
    if (k < 0) {
        if (c->n == c->cap) {
            int64_t nc = 2 * c->cap;
            det_t *nd = (det_t *)realloc(c->d, (size_t)nc * sizeof(det_t));
            if (!nd) return -1;
            c->d = nd;
            double *nv = (double *)realloc(c->v, (size_t)nc * sizeof(double));
            if (!nv) return -1;
            c->v = nv; c->cap = nc;
        }
        k = c->n++;
        c->d[k] = d; c->v[k] = 0.0;
        if (dmap_put(&c->idx, d, k) < 0) return -1;
    }
    c->v[k] += x;
    return 0;
}

/*
 * Definition layer: H_{D',D} for all D' by applying each term of
 * Eq. (general-ham) to |D> literally.  Terms are visited in the order
 * (one-body: Q then P; two-body: R, S, Q, P) and their contributions summed
 * into the entry of the resulting determinant.
 */
static int column_literal_buf(int N, const double *h, const double *g, det_t D, colbuf *out) {
    int M = 2 * N;
    for (int Q = 0; Q < M; Q++) {
        det_t d1 = D; int s1 = annihilate(&d1, N, Q);
        if (!s1) continue;
        for (int P = 0; P < M; P++) {
            double coef = h_so(N, h, P, Q);
            if (coef == 0.0) continue;
            det_t d2 = d1; int s2 = create(&d2, N, P);
            if (!s2) continue;
            if (colbuf_add(out, d2, (double)(s1 * s2) * coef)) return -1;
        }
    }
    for (int R = 0; R < M; R++) {
        det_t d1 = D; int s1 = annihilate(&d1, N, R);          /* a_R acts first */
        if (!s1) continue;
        for (int S = 0; S < M; S++) {
            det_t d2 = d1; int s2 = annihilate(&d2, N, S);     /* then a_S */
            if (!s2) continue;
            for (int Q = 0; Q < M; Q++) {
                det_t d3 = d2; int s3 = create(&d3, N, Q);     /* then a+_Q */
                if (!s3) continue;
                for (int P = 0; P < M; P++) {
                    double v = v_so(N, g, P, Q, R, S);
                    if (v == 0.0) continue;
                    det_t d4 = d3; int s4 = create(&d4, N, P); /* then a+_P */
                    if (!s4) continue;
                    if (colbuf_add(out, d4, 0.5 * (double)(s1 * s2 * s3 * s4) * v)) return -1;
                }
            }
        }
    }
    return 0;
}

/*
 * Eq. (entry) in spin-orbital form.  With sigma the sign of the literal
 * operator product on |D>:
 *   diagonal : sum_{p in occ} h_pp + 1/2 sum_{p,q in occ} (v_pqpq - v_pqqp)
 *   single   : D' = sigma a+_r a_p D,  H = sigma [h_rp + sum_{k in occ(D)} (v_rkpk - v_rkkp)]
 *   double   : D' = sigma a+_r a+_s a_q a_p D (p<q occupied, r<s empty),
 *              H = sigma (v_rspq - v_rsqp)
 * The paper writes the double with annihilators a_p a_q and an unspecified
 * (+-); the operator order a_q a_p used here is the one for which the printed
 * value (v_rspq - v_rsqp) holds with (+-) the literal sign, which the tests
 * confirm against column_literal.
 */
static double diag_sc(int N, const double *h, const double *g, det_t D) {
    int M = 2 * N;
    double e1 = 0.0, e2 = 0.0;
    for (int p = 0; p < M; p++) {
        if (!occupied(&D, N, p)) continue;
        e1 += h_so(N, h, p, p);
        for (int q = 0; q < M; q++) {
            if (!occupied(&D, N, q)) continue;
            e2 += v_so(N, g, p, q, p, q) - v_so(N, g, p, q, q, p);
        }
    }
    return e1 + 0.5 * e2;
}

static int column_sc_buf(int N, const double *h, const double *g, det_t D, colbuf *out) {
    int M = 2 * N;
    if (colbuf_add(out, D, diag_sc(N, h, g, D))) return -1;
    /* singles p -> r, same spin */
    for (int p = 0; p < M; p++) {
        if (!occupied(&D, N, p)) continue;
        for (int r = 0; r < M; r++) {
            if ((r < N) != (p < N)) continue;
            if (occupied(&D, N, r)) continue;
            det_t d = D;
            int s = annihilate(&d, N, p);
            s *= create(&d, N, r);
            double x = h_so(N, h, r, p);
            for (int k = 0; k < M; k++) {
                if (!occupied(&D, N, k)) continue;
                x += v_so(N, g, r, k, p, k) - v_so(N, g, r, k, k, p);
            }
            x *= (double)s;
            if (x != 0.0 && colbuf_add(out, d, x)) return -1;
        }
    }
    /* doubles p<q -> r<s, total spin projection conserved */
    for (int p = 0; p < M; p++) {
        if (!occupied(&D, N, p)) continue;
        for (int q = p + 1; q < M; q++) {
            if (!occupied(&D, N, q)) continue;
            for (int r = 0; r < M; r++) {
                if (occupied(&D, N, r)) continue;
                for (int s = r + 1; s < M; s++) {
                    if (occupied(&D, N, s)) continue;
                    int nb_in = (p >= N) + (q >= N), nb_out = (r >= N) + (s >= N);
                    if (nb_in != nb_out) continue;
                    det_t d = D;
                    int sg = annihilate(&d, N, p);
                    sg *= annihilate(&d, N, q);
                    sg *= create(&d, N, s);
                    sg *= create(&d, N, r);
                    double x = (double)sg * (v_so(N, g, r, s, p, q) - v_so(N, g, r, s, q, p));
                    if (x != 0.0 && colbuf_add(out, d, x)) return -1;
                }
            }
        }
    }
    return 0;
}

/* copy nonzero entries of a column buffer out; returns count or -needed if cap too small */
static int64_t colbuf_emit(const colbuf *c, uint64_t *keys, double *vals, int64_t cap) {
    int64_t n = 0;
    for (int64_t i = 0; i < c->n; i++) if (c->v[i] != 0.0) n++;
    if (n > cap) return -n;
    int64_t k = 0;
    for (int64_t i = 0; i < c->n; i++) {
        if (c->v[i] == 0.0) continue;
        keys[2 * k] = c->d[i].a; keys[2 * k + 1] = c->d[i].b; vals[k] = c->v[i]; k++;
    }
    return n;
}

int64_t orc_column_literal(int N, const double *h, const double *g, uint64_t A, uint64_t B,
                           uint64_t *keys, double *vals, int64_t cap) {
    colbuf c; det_t D = {A, B};
    if (colbuf_init(&c, 1024)) return -1;
    int64_t r = column_literal_buf(N, h, g, D, &c) ? -1 : colbuf_emit(&c, keys, vals, cap);
    colbuf_free(&c);
    return r;
}

int64_t orc_column_sc(int N, const double *h, const double *g, uint64_t A, uint64_t B,
                      uint64_t *keys, double *vals, int64_t cap) {
    colbuf c; det_t D = {A, B};
    if (colbuf_init(&c, 1024)) return -1;
    int64_t r = column_sc_buf(N, h, g, D, &c) ? -1 : colbuf_emit(&c, keys, vals, cap);
    colbuf_free(&c);
    return r;
}

double orc_diag(int N, const double *h, const double *g, uint64_t A, uint64_t B) {
    det_t D = {A, B};
    return diag_sc(N, h, g, D);
}

/* ------------------------------------------------------------------------ */
/* FCI space: enumeration in increasing bitstring order, and ranking         */
/* ------------------------------------------------------------------------ */

static int64_t binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; i++) r = r * (n - k + i) / i;
    return r;
}

/* rank of a bitstring among all strings with the same popcount (colex = numeric order) */
static int64_t string_rank(uint64_t x) {
    int64_t r = 0; int k = 0;
    for (int p = 0; p < 64; p++)
        if ((x >> p) & 1ULL) { k++; r += binom(p, k); }
    return r;
}

/* next bitstring with the same popcount (numeric order) */
static uint64_t next_string(uint64_t x) {
    uint64_t t = x | (x - 1);
    return (t + 1) | (((~t & -~t) - 1) >> (__builtin_ctzll(x) + 1));
}

int64_t orc_fci_dim(int N, int na, int nb) { return binom(N, na) * binom(N, nb); }

/* all determinants, alpha-major: index = rank(A) * C(N, nb) + rank(B) */
int orc_fci_dets(int N, int na, int nb, uint64_t *keys) {
    int64_t da = binom(N, na), db = binom(N, nb);
    uint64_t A = below(na);
    for (int64_t i = 0; i < da; i++) {
        uint64_t B = below(nb);
        for (int64_t j = 0; j < db; j++) {
            keys[2 * (i * db + j)] = A;
            keys[2 * (i * db + j) + 1] = B;
            if (j + 1 < db) B = next_string(B);
        }
        if (i + 1 < da) A = next_string(A);
    }
    return 0;
}

int64_t orc_fci_index(int N, int na, int nb, uint64_t A, uint64_t B) {
    (void)na;
    return string_rank(A) * binom(N, nb) + string_rank(B);
}

/* dense H (dim x dim, row-major H[I*dim+J] = <I|H|J>) from the literal operator */
int orc_dense_H(int N, int na, int nb, const double *h, const double *g, double *H) {
    int64_t dim = orc_fci_dim(N, na, nb);
    uint64_t *keys = (uint64_t *)malloc((size_t)dim * 2 * sizeof(uint64_t));
    if (!keys) return -1;
    orc_fci_dets(N, na, nb, keys);
    memset(H, 0, (size_t)dim * dim * sizeof(double));
    for (int64_t J = 0; J < dim; J++) {
        colbuf c; det_t D = {keys[2 * J], keys[2 * J + 1]};
        if (colbuf_init(&c, 256)) { free(keys); return -1; }
        if (column_literal_buf(N, h, g, D, &c)) { colbuf_free(&c); free(keys); return -1; }
        for (int64_t k = 0; k < c.n; k++) {
            int64_t I = orc_fci_index(N, na, nb, c.d[k].a, c.d[k].b);
            H[I * dim + J] = c.v[k];
        }
        colbuf_free(&c);
    }
    free(keys);
    return 0;
}

/*
 * Sparse H in coordinate form from the Slater-Condon columns (for library
 * eigensolvers on spaces too large for a dense matrix).  Returns the number
 * of nonzeros, or -needed if cap is too small.
 */
int64_t orc_sparse_H(int N, int na, int nb, const double *h, const double *g,
                     int64_t *rows, int64_t *cols, double *vals, int64_t cap) {
    int64_t dim = orc_fci_dim(N, na, nb);
    uint64_t *keys = (uint64_t *)malloc((size_t)dim * 2 * sizeof(uint64_t));
    if (!keys) return -1;
    orc_fci_dets(N, na, nb, keys);
    int64_t nnz = 0;
    for (int64_t J = 0; J < dim; J++) {
        colbuf c; det_t D = {keys[2 * J], keys[2 * J + 1]};
        if (colbuf_init(&c, 256)) { free(keys); return -1; }
        if (column_sc_buf(N, h, g, D, &c)) { colbuf_free(&c); free(keys); return -1; }
        for (int64_t k = 0; k < c.n; k++) {
            if (c.v[k] == 0.0) continue;
            if (nnz < cap) {
                rows[nnz] = orc_fci_index(N, na, nb, c.d[k].a, c.d[k].b);
                cols[nnz] = J; vals[nnz] = c.v[k];
            }
            nnz++;
        }
        colbuf_free(&c);
    }
    free(keys);
    return nnz <= cap ? nnz : -nnz;
}

/* ------------------------------------------------------------------------ */
/* Step size: appendix "Determining Step Size"                               */
/* ------------------------------------------------------------------------ */

/*
 * argmin over eta of h(eta) = eta^4 + v3 eta^3 + v2 eta^2 + v1 eta.
 * The derivative 4 eta^3 + 3 v3 eta^2 + 2 v2 eta + v1 is depressed by
 * eta = x - b/(3a) to x^3 + p x + q; Delta = (q/2)^2 + (p/3)^3.  Delta >= 0:
 * the real root (for Delta = 0 the simple one); Delta < 0: of the three roots
 * x1 < x2 < x3 the one farther from x2, which has the lower value (the quartic
 * differs between x3 and x1 by -(x3 - x1)^3 ((x3 - x2) - (x2 - x1)) / 3); x1
 * on a tie, where a tie is a difference of the two distances below 1e-9 of
 * their sum (a symmetric quartic, e.g. a coordinate that is the only nonzero
 * one, ties exactly, and rounding must not pick a side).  Then Newton on
 * the cubic until the relative change is below 1e-15 (absolute at 0), at most
 * 8 steps.
 */
double orc_line_search(double v1, double v2, double v3) {
    double a = 4.0, b = 3.0 * v3, c = 2.0 * v2, d = v1;
    double p = (3.0 * a * c - b * b) / (3.0 * a * a);
    double q = (2.0 * b * b * b - 9.0 * a * b * c + 27.0 * a * a * d) / (27.0 * a * a * a);
    double delta = (q / 2.0) * (q / 2.0) + (p / 3.0) * (p / 3.0) * (p / 3.0);
    double x;
    if (delta >= 0.0) {
        double sd = sqrt(delta);
        x = cbrt(-q / 2.0 + sd) + cbrt(-q / 2.0 - sd);
    } else {
        double r = 2.0 * sqrt(-p / 3.0);
        double arg = (3.0 * q / (2.0 * p)) * sqrt(-3.0 / p);
        if (arg > 1.0) arg = 1.0;
        if (arg < -1.0) arg = -1.0;
        double th = acos(arg) / 3.0;
        double xs[3];
        const double two_pi = 6.283185307179586476925286766559;
        for (int k = 0; k < 3; k++) xs[k] = r * cos(th - two_pi * k / 3.0);
        /* sort ascending */
        for (int i = 0; i < 3; i++)
            for (int j = i + 1; j < 3; j++)
                if (xs[j] < xs[i]) { double t = xs[i]; xs[i] = xs[j]; xs[j] = t; }
        double d1 = xs[1] - xs[0], d3 = xs[2] - xs[1];
        x = (d3 - d1 > 1e-9 * (d1 + d3)) ? xs[2] : xs[0];
    }
    double eta = x - b / (3.0 * a);
    for (int it = 0; it < 8; it++) {
        double f = ((4.0 * eta + 3.0 * v3) * eta + 2.0 * v2) * eta + v1;
        double fp = (12.0 * eta + 6.0 * v3) * eta + 2.0 * v2;
        if (fp == 0.0) break;
        double nxt = eta - f / fp;
        double ch = fabs(nxt - eta);
        double sc = fabs(eta);
        eta = nxt;
        if (sc == 0.0 ? ch < 1e-300 : ch / sc < 1e-15) break;
    }
    return eta;
}

/* ------------------------------------------------------------------------ */
/* Small symmetric eigensolver: cyclic Jacobi (Golub & Van Loan, Sec. 8.5)   */
/* ------------------------------------------------------------------------ */

/* A (n x n, row-major, symmetric) is destroyed; w = eigenvalues, V columns = eigenvectors */
static void jacobi_eig(int n, double *A, double *w, double *V) {
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) {
                tot += A[i * n + j] * A[i * n + j];
                if (i != j) off += A[i * n + j] * A[i * n + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double app = A[p * n + p], aqq = A[q * n + q];
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
                for (int k = 0; k < n; k++) {   /* A <- A J */
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = cs * akp - sn * akq;
                    A[k * n + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; k++) {   /* A <- J^T A */
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = cs * apk - sn * aqk;
                    A[q * n + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < n; k++) {   /* V <- V J */
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = cs * vkp - sn * vkq;
                    V[k * n + q] = sn * vkp + cs * vkq;
                }
            }
    }
    for (int i = 0; i < n; i++) w[i] = A[i * n + i];
}

int orc_sym_eig(int n, const double *A, double *w, double *V) {
    double *T = (double *)malloc((size_t)n * n * sizeof(double));
    if (!T) return -1;
    memcpy(T, A, (size_t)n * n * sizeof(double));
    jacobi_eig(n, T, w, V);
    free(T);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithms 1 and 2                                                         */
/* ------------------------------------------------------------------------ */

typedef struct {
    int N, na, nb, m;
    const double *h, *g;           /* borrowed; caller keeps them alive */
    double tau;
    /* sparse c and b: map det -> entry index; entries grow, never removed */
    dmap map;
    int64_t n, cap;
    det_t *key;
    double *c, *b;
    /* c^T c and c^T H c in binary128 */
    quad mu, alpha;
    double dx, theta;
    int64_t iter;
    /* candidate list: entry indices of the last processed columns, deduplicated */
    int64_t ncand, candcap;
    int64_t *cand;
    /* statistics */
    int64_t elements, applied, dropped;
    int64_t last_m;
    int64_t *last_sel;             /* entry indices selected in the last step */
    double last_eta[4096];
    int degenerate_steps;
} orc_state;

static int64_t st_entry(orc_state *st, det_t d, int insert) {
    int64_t k = dmap_get(&st->map, d);
    if (k >= 0 || !insert) return k;
    if (st->n == st->cap) {
        int64_t nc = 2 * st->cap;
        det_t *nk = (det_t *)realloc(st->key, (size_t)nc * sizeof(det_t));
        if (!nk) return -2;
        st->key = nk;
        double *ncc = (double *)realloc(st->c, (size_t)nc * sizeof(double));
        if (!ncc) return -2;
        st->c = ncc;
        double *nbb = (double *)realloc(st->b, (size_t)nc * sizeof(double));
        if (!nbb) return -2;
        st->b = nbb; st->cap = nc;
    }
    k = st->n++;
    st->key[k] = d; st->c[k] = 0.0; st->b[k] = 0.0;
    if (dmap_put(&st->map, d, k) < 0) return -2;
    return k;
}

static int cand_push(orc_state *st, int64_t k) {
    if (st->ncand == st->candcap) {
        int64_t nc = 2 * st->candcap;
        int64_t *p = (int64_t *)realloc(st->cand, (size_t)nc * sizeof(int64_t));
        if (!p) return -1;
        st->cand = p; st->candcap = nc;
    }
    st->cand[st->ncand++] = k;
    return 0;
}

/*
 * Add eta_i * H_{:,i} to b with the compression rule (Sec. on CDFCI): b_j is
 * updated only if c_j != 0 or |eta_i H_ji| >= tau; an absent j is inserted
 * only in the second case.  Updated entries become candidates.  Also returns
 * sum_j H_ji c_j over the column (using c as it is now) for the recalculation
 * of b_i (Eq. recalculate-b).
 */
static int scatter_column(orc_state *st, det_t Di, double eta, double *recalc, dmap *seen) {
    colbuf col;
    if (colbuf_init(&col, 1024)) return -1;
    if (column_sc_buf(st->N, st->h, st->g, Di, &col)) { colbuf_free(&col); return -1; }
    double acc = 0.0;
    for (int64_t t = 0; t < col.n; t++) {
        double Hji = col.v[t];
        if (Hji == 0.0) continue;
        st->elements++;
        det_t dj = col.d[t];
        int64_t k = st_entry(st, dj, 0);
        double cj = (k >= 0) ? st->c[k] : 0.0;
        double upd = eta * Hji;
        if (cj != 0.0 || fabs(upd) >= st->tau) {
            if (k < 0) { k = st_entry(st, dj, 1); if (k < 0) { colbuf_free(&col); return -1; } }
            st->b[k] += upd;
            st->applied++;
            if (dmap_get(seen, dj) < 0) { dmap_put(seen, dj, k); if (cand_push(st, k)) { colbuf_free(&col); return -1; } }
        } else {
            st->dropped++;
        }
        acc += Hji * cj;
    }
    colbuf_free(&col);
    *recalc = acc;
    return 0;
}

static double grad_abs(const orc_state *st, int64_t k) {
    double mu = (double)st->mu;
    return fabs(4.0 * st->b[k] + 4.0 * mu * st->c[k]);
}

/* candidate order: larger |g| first, then smaller key */
static const orc_state *g_sort_state;
static int cand_cmp(const void *x, const void *y) {
    int64_t i = *(const int64_t *)x, j = *(const int64_t *)y;
    double gi = grad_abs(g_sort_state, i), gj = grad_abs(g_sort_state, j);
    if (gi > gj) return -1;
    if (gi < gj) return 1;
    if (det_less(g_sort_state->key[i], g_sort_state->key[j])) return -1;
    if (det_less(g_sort_state->key[j], g_sort_state->key[i])) return 1;
    return 0;
}

orc_state *orc_create(int N, int na, int nb, const double *h, const double *g,
                      uint64_t refA, uint64_t refB, double tau, int m, double theta) {
    if (N < 1 || N > 64 || na < 0 || nb < 0 || na > N || nb > N || m < 1 || m > 4096) return NULL;
    orc_state *st = (orc_state *)calloc(1, sizeof(orc_state));
    if (!st) return NULL;
    st->N = N; st->na = na; st->nb = nb; st->m = m; st->h = h; st->g = g; st->tau = tau;
    st->theta = theta;
    st->cap = 1024;
    st->key = (det_t *)malloc((size_t)st->cap * sizeof(det_t));
    st->c = (double *)malloc((size_t)st->cap * sizeof(double));
    st->b = (double *)malloc((size_t)st->cap * sizeof(double));
    st->candcap = 1024;
    st->cand = (int64_t *)malloc((size_t)st->candcap * sizeof(int64_t));
    st->last_sel = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    if (!st->key || !st->c || !st->b || !st->cand || !st->last_sel || dmap_init(&st->map, 1024)) return NULL;
    /* reference determinant: given, or aufbau on h_pp (smallest first, ties to lower index) */
    if (refA == 0 && refB == 0) {
        int order[64];
        for (int p = 0; p < N; p++) order[p] = p;
        for (int i = 0; i < N; i++)
            for (int j = i + 1; j < N; j++) {
                double hi = h[order[i] * N + order[i]], hj = h[order[j] * N + order[j]];
                if (hj < hi || (hj == hi && order[j] < order[i])) { int t = order[i]; order[i] = order[j]; order[j] = t; }
            }
        for (int k = 0; k < na; k++) refA |= 1ULL << order[k];
        for (int k = 0; k < nb; k++) refB |= 1ULL << order[k];
    }
    /* Initialisation of Algorithms 1 and 2: c = e_ref, b = H c (with the
       compression rule), mu = 1, alpha = H_ref,ref; candidates = column(ref). */
    det_t ref = {refA, refB};
    int64_t kr = st_entry(st, ref, 1);
    st->c[kr] = 1.0;
    dmap seen; dmap_init(&seen, 1024);
    double rc;
    if (scatter_column(st, ref, 1.0, &rc, &seen)) return NULL;
    st->b[kr] = rc;
    if (dmap_get(&seen, ref) < 0) cand_push(st, kr);
    dmap_free(&seen);
    st->mu = 1;
    st->alpha = (quad)diag_sc(N, h, g, ref);
    st->dx = 0.0;
    st->iter = 0;
    return st;
}

/*
 * Start vector (the reading behind cdfci_set_initial): clear the state, then
 * for each entry k in order take coordinate D_k from its current value with
 * the step fixed to c_k, exactly as the initialisation above takes e_ref with
 * step 1: c_k += c_k's step, b += step H_{:,k} with the compression rule,
 * b_k recalculated, mu and alpha by Eq. (update-var) with the pre-update c_k,
 * b_k.  No iteration is counted.  m = 1: the candidates are those of the last
 * start column (as after any step); m > 1: of every start column,
 * deduplicated.  Returns 0, -1 (allocation) or -4 (a repeated key).
 */
int orc_set_initial(orc_state *st, const uint64_t *keys, const double *c, int64_t n) {
    dmap_free(&st->map);
    if (dmap_init(&st->map, 1024)) return -1;
    st->n = 0; st->ncand = 0;
    st->mu = 0; st->alpha = 0; st->dx = 0.0; st->iter = 0;
    st->elements = 0; st->applied = 0; st->dropped = 0; st->last_m = 0;
    dmap seen;
    if (dmap_init(&seen, 1024)) return -1;
    for (int64_t k = 0; k < n; k++) {
        det_t Di = {keys[2 * k], keys[2 * k + 1]};
        if (st_entry(st, Di, 0) >= 0 && st->c[st_entry(st, Di, 0)] != 0.0) { dmap_free(&seen); return -4; }
        int64_t kk = st_entry(st, Di, 1);
        if (kk < 0) { dmap_free(&seen); return -1; }
        double ci = st->c[kk], bi = st->b[kk];
        double Hii = diag_sc(st->N, st->h, st->g, Di);
        double eta = c[k];
        st->c[kk] = ci + eta;
        if (st->m == 1) {                  /* candidates: the last processed column only */
            st->ncand = 0;
            dmap_free(&seen);
            if (dmap_init(&seen, 1024)) return -1;
        }
        double rc;
        if (scatter_column(st, Di, eta, &rc, &seen)) { dmap_free(&seen); return -1; }
        if (dmap_get(&seen, Di) < 0) { dmap_put(&seen, Di, kk); if (cand_push(st, kk)) { dmap_free(&seen); return -1; } }
        st->b[kk] = rc;
        st->mu = st->mu + (quad)2.0 * (quad)eta * (quad)ci + (quad)eta * (quad)eta;
        st->alpha = st->alpha + (quad)2.0 * (quad)eta * (quad)bi + (quad)eta * (quad)eta * (quad)Hii;
    }
    dmap_free(&seen);
    return 0;
}

void orc_destroy(orc_state *st) {
    if (!st) return;
    dmap_free(&st->map);
    free(st->key); free(st->c); free(st->b); free(st->cand); free(st->last_sel);
    free(st);
}

/* one iteration of Algorithm 1 (m = 1) */
static int step_cd(orc_state *st) {
    /* select: argmax over the candidates of |4 b_i + 4 mu c_i| */
    int64_t best = -1;
    for (int64_t t = 0; t < st->ncand; t++) {
        int64_t k = st->cand[t];
        if (best < 0) { best = k; continue; }
        double gk = grad_abs(st, k), gb = grad_abs(st, best);
        if (gk > gb || (gk == gb && det_less(st->key[k], st->key[best]))) best = k;
    }
    if (best < 0) return -3;
    det_t Di = st->key[best];
    double ci = st->c[best], bi = st->b[best];
    double mu = (double)st->mu;
    double Hii = diag_sc(st->N, st->h, st->g, Di);
    /* step size from the cubic (appendix) */
    double v1 = 4.0 * bi + 4.0 * mu * ci;
    double v2 = 2.0 * Hii + 4.0 * ci * ci + 2.0 * mu;
    double v3 = 4.0 * ci;
    double eta = orc_line_search(v1, v2, v3);
    /* update c_i; b += eta H_{:,i} with compression; recalculate b_i */
    st->c[best] = ci + eta;
    st->ncand = 0;
    dmap seen; dmap_init(&seen, 1024);
    double rc;
    if (scatter_column(st, Di, eta, &rc, &seen)) { dmap_free(&seen); return -1; }
    if (dmap_get(&seen, Di) < 0) cand_push(st, best);
    dmap_free(&seen);
    st->b[best] = rc;
    /* mu and alpha with the pre-update c_i, b_i (Eq. update-var) */
    st->mu = st->mu + (quad)2.0 * (quad)eta * (quad)ci + (quad)eta * (quad)eta;
    st->alpha = st->alpha + (quad)2.0 * (quad)eta * (quad)bi + (quad)eta * (quad)eta * (quad)Hii;
    st->dx = st->theta * st->dx + (1.0 - st->theta) * fabs(eta);
    st->last_m = 1; st->last_sel[0] = best; st->last_eta[0] = eta;
    st->iter++;
    return 0;
}

/* H_{I_a, I_b} for the selected block from the Slater-Condon columns */
static int block_H(orc_state *st, int64_t m, const int64_t *sel, double *HII) {
    dmap pos; dmap_init(&pos, 2 * m + 2);
    for (int64_t a = 0; a < m; a++) dmap_put(&pos, st->key[sel[a]], a);
    memset(HII, 0, (size_t)m * m * sizeof(double));
    for (int64_t bcol = 0; bcol < m; bcol++) {
        colbuf col;
        if (colbuf_init(&col, 1024)) { dmap_free(&pos); return -1; }
        if (column_sc_buf(st->N, st->h, st->g, st->key[sel[bcol]], &col)) { colbuf_free(&col); dmap_free(&pos); return -1; }
        for (int64_t t = 0; t < col.n; t++) {
            int64_t a = dmap_get(&pos, col.d[t]);
            if (a >= 0) HII[a * m + bcol] = col.v[t];
        }
        colbuf_free(&col);
    }
    dmap_free(&pos);
    return 0;
}

/* one iteration of Algorithm 2 (m >= 1 block update with scaling factor gamma) */
static int step_mcd(orc_state *st) {
    if (st->ncand == 0) return -3;
    /* select: the m largest |4 b_i + 4 mu c_i| among the deduplicated candidates */
    g_sort_state = st;
    qsort(st->cand, (size_t)st->ncand, sizeof(int64_t), cand_cmp);
    int64_t m = st->ncand < st->m ? st->ncand : st->m;
    int64_t *sel = st->last_sel;
    for (int64_t a = 0; a < m; a++) sel[a] = st->cand[a];
    double *HII = (double *)malloc((size_t)m * m * sizeof(double));
    double *cI = (double *)malloc((size_t)m * sizeof(double));
    double *bI = (double *)malloc((size_t)m * sizeof(double));
    int64_t n1 = m + 1;
    double *R = (double *)malloc((size_t)n1 * n1 * sizeof(double));
    double *w = (double *)malloc((size_t)n1 * sizeof(double));
    double *V = (double *)malloc((size_t)n1 * n1 * sizeof(double));
    double *eta = (double *)malloc((size_t)m * sizeof(double));
    if (!HII || !cI || !bI || !R || !w || !V || !eta) return -1;
    if (block_H(st, m, sel, HII)) return -1;
    quad cc = 0;
    int64_t nnz_in = 0, nnz_all = 0;
    for (int64_t a = 0; a < m; a++) {
        cI[a] = st->c[sel[a]]; bI[a] = st->b[sel[a]];
        cc += (quad)cI[a] * (quad)cI[a];
        if (cI[a] != 0.0) nnz_in++;
    }
    for (int64_t k = 0; k < st->n; k++) if (st->c[k] != 0.0) nnz_all++;
    /* nu = ||c - E_I c_I||; zero exactly when c has no support outside I */
    int degenerate = (nnz_all == nnz_in);
    quad nu2 = st->mu - cc;
    double nu = degenerate ? 0.0 : (double)sqrtl((long double)(nu2 > 0 ? nu2 : 0));
    double gamma;
    if (!degenerate && nu > 0.0) {
        /* reduced matrix R = Q^T H Q with Q = [c~, E_I] */
        quad cHc = 0, cb = 0;
        for (int64_t a = 0; a < m; a++) {
            quad t = 0;
            for (int64_t bb = 0; bb < m; bb++) t += (quad)HII[a * m + bb] * (quad)cI[bb];
            cHc += (quad)cI[a] * t;
            cb += (quad)cI[a] * (quad)bI[a];
            R[0 * n1 + (a + 1)] = R[(a + 1) * n1 + 0] = (double)(((quad)bI[a] - t) / (quad)nu);
        }
        R[0] = (double)((st->alpha - 2 * cb + cHc) / ((quad)nu * (quad)nu));
        for (int64_t a = 0; a < m; a++)
            for (int64_t bb = 0; bb < m; bb++) R[(a + 1) * n1 + (bb + 1)] = HII[a * m + bb];
        orc_sym_eig((int)n1, R, w, V);
        int64_t lo = 0;
        for (int64_t k = 1; k < n1; k++) if (w[k] < w[lo]) lo = k;
        double lam = w[lo];
        if (!(lam < 0.0)) return -4;
        double sc = sqrt(-lam);
        double z0 = sc * V[0 * n1 + lo];
        double sgn = 1.0;
        if (z0 < 0.0) sgn = -1.0;
        else if (z0 == 0.0) {
            double dot = 0.0;
            for (int64_t a = 0; a < m; a++) dot += V[(a + 1) * n1 + lo] * cI[a];
            if (dot < 0.0) sgn = -1.0;
        }
        /* z = [nu gamma; c_I gamma + eta] (Eq. def-z) */
        gamma = sgn * z0 / nu;
        for (int64_t a = 0; a < m; a++) eta[a] = sgn * sc * V[(a + 1) * n1 + lo] - gamma * cI[a];
    } else {
        /* c lies in span(E_I): solve the m x m problem on H_II, gamma = 1 */
        st->degenerate_steps++;
        double *Hc = (double *)malloc((size_t)m * m * sizeof(double));
        double *wm = (double *)malloc((size_t)m * sizeof(double));
        double *Vm = (double *)malloc((size_t)m * m * sizeof(double));
        memcpy(Hc, HII, (size_t)m * m * sizeof(double));
        orc_sym_eig((int)m, Hc, wm, Vm);
        int64_t lo = 0;
        for (int64_t k = 1; k < m; k++) if (wm[k] < wm[lo]) lo = k;
        if (!(wm[lo] < 0.0)) return -4;
        double sc = sqrt(-wm[lo]);
        double dot = 0.0;
        for (int64_t a = 0; a < m; a++) dot += Vm[a * m + lo] * cI[a];
        double sgn = dot < 0.0 ? -1.0 : 1.0;
        gamma = 1.0;
        for (int64_t a = 0; a < m; a++) eta[a] = sgn * sc * Vm[a * m + lo] - cI[a];
        free(Hc); free(wm); free(Vm);
    }
    /* scalars with the pre-update c_I, b_I */
    quad etc = 0, etb = 0, ete = 0, eHe = 0;
    for (int64_t a = 0; a < m; a++) {
        etc += (quad)eta[a] * (quad)cI[a];
        etb += (quad)eta[a] * (quad)bI[a];
        ete += (quad)eta[a] * (quad)eta[a];
        quad t = 0;
        for (int64_t bb = 0; bb < m; bb++) t += (quad)HII[a * m + bb] * (quad)eta[bb];
        eHe += (quad)eta[a] * t;
    }
    quad G = (quad)gamma;
    st->mu = G * G * st->mu + 2 * G * etc + ete;
    st->alpha = G * G * st->alpha + 2 * G * etb + eHe;
    /* c <- gamma c + E_I eta ; b <- gamma b (then + H_{:,I} eta below) */
    if (gamma != 1.0)
        for (int64_t k = 0; k < st->n; k++) { st->c[k] *= gamma; st->b[k] *= gamma; }
    for (int64_t a = 0; a < m; a++) st->c[sel[a]] += eta[a];
    /* b += H_{:,I} eta with compression; candidates = union of the columns */
    st->ncand = 0;
    dmap seen; dmap_init(&seen, 4096);
    double *rc = (double *)malloc((size_t)m * sizeof(double));
    for (int64_t a = 0; a < m; a++) {
        if (scatter_column(st, st->key[sel[a]], eta[a], &rc[a], &seen)) return -1;
    }
    /* recalculation of b_I needs the final c (all columns' c reads above used
       the updated c already, since c is not touched by the scatter) */
    for (int64_t a = 0; a < m; a++) {
        st->b[sel[a]] = rc[a];
        if (dmap_get(&seen, st->key[sel[a]]) < 0) { dmap_put(&seen, st->key[sel[a]], sel[a]); cand_push(st, sel[a]); }
    }
    dmap_free(&seen);
    double nrm = 0.0;
    for (int64_t a = 0; a < m; a++) nrm += eta[a] * eta[a];
    st->dx = st->theta * st->dx + (1.0 - st->theta) * sqrt(nrm);
    st->last_m = m;
    for (int64_t a = 0; a < m && a < 4096; a++) st->last_eta[a] = eta[a];
    st->iter++;
    free(HII); free(cI); free(bI); free(R); free(w); free(V); free(eta); free(rc);
    return 0;
}

int orc_step(orc_state *st, int64_t n_iter) {
    for (int64_t i = 0; i < n_iter; i++) {
        int r = (st->m == 1) ? step_cd(st) : step_mcd(st);
        if (r) return r;
    }
    return 0;
}

/* energy = alpha / mu (Rayleigh quotient of c) */
double orc_energy(const orc_state *st) { return (double)(st->alpha / st->mu); }

/* out: mu, alpha, dx, iterations, n_entries, nnz_c, elements, applied, dropped, degenerate_steps */
void orc_info(const orc_state *st, double *out) {
    int64_t nnz = 0;
    for (int64_t k = 0; k < st->n; k++) if (st->c[k] != 0.0) nnz++;
    out[0] = (double)st->mu; out[1] = (double)st->alpha; out[2] = st->dx; out[3] = (double)st->iter;
    out[4] = (double)st->n; out[5] = (double)nnz; out[6] = (double)st->elements;
    out[7] = (double)st->applied; out[8] = (double)st->dropped; out[9] = (double)st->degenerate_steps;
}

/* stored entries (key, c, b); returns count, or -count if cap is too small */
int64_t orc_export(const orc_state *st, uint64_t *keys, double *c, double *b, int64_t cap) {
    if (st->n > cap) return -st->n;
    for (int64_t k = 0; k < st->n; k++) {
        keys[2 * k] = st->key[k].a; keys[2 * k + 1] = st->key[k].b; c[k] = st->c[k]; b[k] = st->b[k];
    }
    return st->n;
}

/* keys and step sizes selected in the last iteration; returns m */
int64_t orc_last_step(const orc_state *st, uint64_t *keys, double *eta, int64_t cap) {
    int64_t m = st->last_m;
    for (int64_t a = 0; a < m && a < cap; a++) {
        keys[2 * a] = st->key[st->last_sel[a]].a;
        keys[2 * a + 1] = st->key[st->last_sel[a]].b;
        eta[a] = st->last_eta[a];
    }
    return m;
}

/* current candidate keys (deduplicated union of the last processed columns) */
int64_t orc_candidates(const orc_state *st, uint64_t *keys, int64_t cap) {
    if (st->ncand > cap) return -st->ncand;
    for (int64_t t = 0; t < st->ncand; t++) {
        keys[2 * t] = st->key[st->cand[t]].a; keys[2 * t + 1] = st->key[st->cand[t]].b;
    }
    return st->ncand;
}

/* ------------------------------------------------------------------------ */
/* Reduced density matrices (Sec. "Optimal Orbital Selections")              */
/* ------------------------------------------------------------------------ */

/*
 * Spin-summed RDMs of Psi = sum_J c_J |J>, normalised by c.c:
 *   gamma[p][q]       = sum_s  <Psi| a+_{p s} a_{q s} |Psi>
 *   Gamma[p][q][r][s] = sum_{s,t} <Psi| a+_{p s} a+_{r t} a_{s t} a_{q s} |Psi>
 * (chemists' index order: E = sum h_pq gamma_pq + 1/2 sum (pq|rs) Gamma_pqrs,
 * which is Eq. (general-ham) with v_{PQRS} = (pr|qs)).  Operators are applied
 * literally to each |J>, right to left; the result is projected on <I|.
 */
int orc_rdm(int N, int64_t n, const uint64_t *keys, const double *c, double *g1, double *g2) {
    dmap pos;
    if (dmap_init(&pos, n + 1)) return -1;
    double norm = 0.0;
    for (int64_t k = 0; k < n; k++) {
        det_t d = {keys[2 * k], keys[2 * k + 1]};
        dmap_put(&pos, d, k);
        norm += c[k] * c[k];
    }
    memset(g1, 0, (size_t)N * N * sizeof(double));
    memset(g2, 0, (size_t)N * N * N * N * sizeof(double));
    for (int64_t J = 0; J < n; J++) {
        if (c[J] == 0.0) continue;
        det_t DJ = {keys[2 * J], keys[2 * J + 1]};
        for (int sg = 0; sg < 2; sg++) {
            for (int q = 0; q < N; q++) {
                det_t d1 = DJ; int s1 = annihilate(&d1, N, q + sg * N);
                if (!s1) continue;
                for (int p = 0; p < N; p++) {
                    det_t d2 = d1; int s2 = create(&d2, N, p + sg * N);
                    if (!s2) continue;
                    int64_t I = dmap_get(&pos, d2);
                    if (I >= 0) g1[p * N + q] += c[I] * c[J] * (double)(s1 * s2);
                }
                for (int tg = 0; tg < 2; tg++)
                    for (int s = 0; s < N; s++) {
                        det_t d2 = d1; int s2 = annihilate(&d2, N, s + tg * N);
                        if (!s2) continue;
                        for (int r = 0; r < N; r++) {
                            det_t d3 = d2; int s3 = create(&d3, N, r + tg * N);
                            if (!s3) continue;
                            for (int p = 0; p < N; p++) {
                                det_t d4 = d3; int s4 = create(&d4, N, p + sg * N);
                                if (!s4) continue;
                                int64_t I = dmap_get(&pos, d4);
                                if (I >= 0)
                                    g2[(((size_t)p * N + q) * N + r) * N + s] += c[I] * c[J] * (double)(s1 * s2 * s3 * s4);
                            }
                        }
                    }
            }
        }
    }
    for (int64_t k = 0; k < (int64_t)N * N; k++) g1[k] /= norm;
    for (int64_t k = 0; k < (int64_t)N * N * N * N; k++) g2[k] /= norm;
    dmap_free(&pos);
    return 0;
}

/*
 * Algorithm 1 step whose coordinate is given (for comparing runs whose
 * argmax differs only at exact ties of |4 b + 4 mu c|).  On return g_choice
 * is |4 b_i + 4 mu c_i| of the given coordinate and g_max the largest over the
 * candidates, both before the step; returns -5 if the key is not a candidate.
 */
int orc_step_choice(orc_state *st, uint64_t A, uint64_t B, double *g_choice, double *g_max) {
    if (st->m != 1) return -1;
    det_t want = {A, B};
    int64_t pick = -1;
    double gm = 0.0;
    for (int64_t t = 0; t < st->ncand; t++) {
        int64_t k = st->cand[t];
        double gk = grad_abs(st, k);
        if (gk > gm) gm = gk;
        if (st->key[k].a == want.a && st->key[k].b == want.b) pick = k;
    }
    *g_max = gm;
    if (pick < 0) return -5;
    *g_choice = grad_abs(st, pick);
    /* move the chosen candidate to the front and run the usual step on a
       one-element candidate list */
    st->cand[0] = pick;
    st->ncand = 1;
    return step_cd(st);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 3 (xCDFCI): K + 1 states, one row of C per step                  */
/* ------------------------------------------------------------------------ */
/*
 * State: rows C_{D,:}, B_{D,:} = (H C)_{D,:} (k1 = K + 1 values each), the
 * (k1 x k1) matrices S = C^T C and M = C^T H C in binary128, the candidate
 * list.  Readings (the paper leaves them open):
 *   - start: C = [e_{D_0} ... e_{D_K}] for k1 given determinants, built as k1
 *     forced row steps (row D_k += 1 * e_k) in order, each column scattered
 *     with the compression rule; candidates afterwards = every start column;
 *   - compression of B rows: row j is updated iff some C_{j,k} != 0 or
 *     max_k |eta H_ji g_k| >= tau (an absent row only in the second case);
 *   - h'(0) = <G, e_i g> = ||G_i||^2 (G = 4B + 4CS already holds the factor 4):
 *     w1 = ||g||^2, and the eta^2 terms of the S and M updates are the outer
 *     product g^T g;
 *   - candidates after a step: the rows the column updated, plus i;
 *   - ties of ||G_i||_inf: the smaller key; dx <- theta dx + (1 - theta) |eta| ||g||_2.
 */
#define XK_MAX 8
typedef struct {
    int N, na, nb, k1;
    const double *h, *g;
    double tau, theta;
    dmap map;
    int64_t n, cap;
    det_t *key;
    double *C, *B;                 /* n x k1 each */
    quad S[XK_MAX * XK_MAX], M[XK_MAX * XK_MAX];
    double dx;
    int64_t iter, elements, applied, dropped;
    int64_t ncand, candcap;
    int64_t *cand;
    det_t last_key;
    double last_eta;
} orx_state;

static int64_t orx_entry(orx_state *st, det_t d, int insert) {
    int64_t k = dmap_get(&st->map, d);
    if (k >= 0 || !insert) return k;
    if (st->n == st->cap) {
        int64_t nc = 2 * st->cap;
        det_t *nk = (det_t *)realloc(st->key, (size_t)nc * sizeof(det_t));
        if (!nk) return -2;
        st->key = nk;
        double *ncc = (double *)realloc(st->C, (size_t)nc * st->k1 * sizeof(double));
        if (!ncc) return -2;
        st->C = ncc;
        double *nbb = (double *)realloc(st->B, (size_t)nc * st->k1 * sizeof(double));
        if (!nbb) return -2;
        st->B = nbb; st->cap = nc;
    }
    k = st->n++;
    st->key[k] = d;
    for (int a = 0; a < st->k1; a++) { st->C[k * st->k1 + a] = 0.0; st->B[k * st->k1 + a] = 0.0; }
    if (dmap_put(&st->map, d, k) < 0) return -2;
    return k;
}

static int orx_cand_push(orx_state *st, int64_t k) {
    if (st->ncand == st->candcap) {
        int64_t nc = 2 * st->candcap;
        int64_t *p = (int64_t *)realloc(st->cand, (size_t)nc * sizeof(int64_t));
        if (!p) return -1;
        st->cand = p; st->candcap = nc;
    }
    st->cand[st->ncand++] = k;
    return 0;
}

/* B += H_{:,i} w (w = eta g, k1 values) with the row compression rule; recalc = sum_j H_ji C_{j,:} */
static int orx_scatter(orx_state *st, det_t Di, const double *w, double *recalc, dmap *seen) {
    const int k1 = st->k1;
    colbuf col;
    if (colbuf_init(&col, 1024)) return -1;
    if (column_sc_buf(st->N, st->h, st->g, Di, &col)) { colbuf_free(&col); return -1; }
    for (int a = 0; a < k1; a++) recalc[a] = 0.0;
    for (int64_t t = 0; t < col.n; t++) {
        double Hji = col.v[t];
        if (Hji == 0.0) continue;
        st->elements++;
        det_t dj = col.d[t];
        int64_t k = orx_entry(st, dj, 0);
        int cnz = 0;
        double vmax = 0.0;
        double upd[XK_MAX];
        for (int a = 0; a < k1; a++) {
            upd[a] = Hji * w[a];
            if (fabs(upd[a]) > vmax) vmax = fabs(upd[a]);
            if (k >= 0 && st->C[k * k1 + a] != 0.0) cnz = 1;
        }
        if (cnz || vmax >= st->tau) {
            if (k < 0) { k = orx_entry(st, dj, 1); if (k < 0) { colbuf_free(&col); return -1; } }
            for (int a = 0; a < k1; a++) st->B[k * k1 + a] += upd[a];
            st->applied++;
            if (dmap_get(seen, dj) < 0) { dmap_put(seen, dj, k); if (orx_cand_push(st, k)) { colbuf_free(&col); return -1; } }
        } else {
            st->dropped++;
        }
        if (k >= 0)
            for (int a = 0; a < k1; a++) recalc[a] += Hji * st->C[k * k1 + a];
    }
    colbuf_free(&col);
    return 0;
}

/* the row update C_i += eta g with its column, the recalculated B_i and the S, M updates */
static int orx_row_step(orx_state *st, det_t Di, double eta, const double *g, dmap *seen) {
    const int k1 = st->k1;
    int64_t i = orx_entry(st, Di, 1);
    if (i < 0) return -1;
    double c[XK_MAX], b[XK_MAX], w[XK_MAX], rc[XK_MAX];
    for (int a = 0; a < k1; a++) { c[a] = st->C[i * k1 + a]; b[a] = st->B[i * k1 + a]; w[a] = eta * g[a]; }
    double Hii = diag_sc(st->N, st->h, st->g, Di);
    for (int a = 0; a < k1; a++)
        for (int bb = 0; bb < k1; bb++) {
            quad ga = (quad)g[a], gb = (quad)g[bb], e = (quad)eta;
            st->S[a * k1 + bb] += e * ((quad)c[a] * gb + ga * (quad)c[bb]) + e * e * ga * gb;
            st->M[a * k1 + bb] += e * ((quad)b[a] * gb + ga * (quad)b[bb]) + e * e * (quad)Hii * ga * gb;
        }
    for (int a = 0; a < k1; a++) st->C[i * k1 + a] = c[a] + w[a];
    if (orx_scatter(st, Di, w, rc, seen)) return -1;
    i = orx_entry(st, Di, 0);
    for (int a = 0; a < k1; a++) st->B[i * k1 + a] = rc[a];
    if (dmap_get(seen, Di) < 0) { dmap_put(seen, Di, i); if (orx_cand_push(st, i)) return -1; }
    st->last_key = Di; st->last_eta = eta;
    return 0;
}

/*
 * Coefficients w1..w4 of h(eta) = f(C + eta e_i g) - f(C) (appendix
 * "Determining Step Size", problem choose-eta) from the row c = C_i, g, S and
 * H_ii; w[0] is set to 0 (f(C) itself is not needed).
 */
void orx_quartic(int k1, const double *c, const double *g, const double *S, double Hii, double *w) {
    double gg = 0.0, cg = 0.0, cc = 0.0, gSg = 0.0;
    for (int a = 0; a < k1; a++) {
        gg += g[a] * g[a]; cg += c[a] * g[a]; cc += c[a] * c[a];
        for (int b = 0; b < k1; b++) gSg += g[a] * S[a * k1 + b] * g[b];
    }
    w[0] = 0.0;
    w[1] = gg;
    w[2] = 2.0 * Hii * gg + 2.0 * cg * cg + 2.0 * cc * gg + 2.0 * gSg;
    w[3] = 4.0 * gg * cg;
    w[4] = gg * gg;
}

orx_state *orx_create(int N, int na, int nb, const double *h, const double *g, const uint64_t *keys, int k1,
                      double tau, double theta) {
    if (N < 1 || N > 64 || k1 < 1 || k1 > XK_MAX) return NULL;
    orx_state *st = (orx_state *)calloc(1, sizeof(orx_state));
    if (!st) return NULL;
    st->N = N; st->na = na; st->nb = nb; st->k1 = k1; st->h = h; st->g = g; st->tau = tau; st->theta = theta;
    st->cap = 1024;
    st->key = (det_t *)malloc((size_t)st->cap * sizeof(det_t));
    st->C = (double *)malloc((size_t)st->cap * k1 * sizeof(double));
    st->B = (double *)malloc((size_t)st->cap * k1 * sizeof(double));
    st->candcap = 1024;
    st->cand = (int64_t *)malloc((size_t)st->candcap * sizeof(int64_t));
    if (!st->key || !st->C || !st->B || !st->cand || dmap_init(&st->map, 1024)) return NULL;
    dmap seen;
    if (dmap_init(&seen, 1024)) return NULL;
    for (int k = 0; k < k1; k++) {
        det_t D = {keys[2 * k], keys[2 * k + 1]};
        double e[XK_MAX];
        for (int a = 0; a < k1; a++) e[a] = (a == k) ? 1.0 : 0.0;
        if (orx_entry(st, D, 0) >= 0) {
            int nz = 0;
            int64_t q = orx_entry(st, D, 0);
            for (int a = 0; a < k1; a++) nz |= st->C[q * k1 + a] != 0.0;
            if (nz) { dmap_free(&seen); return NULL; }       /* a repeated start determinant */
        }
        if (orx_row_step(st, D, 1.0, e, &seen)) { dmap_free(&seen); return NULL; }
    }
    dmap_free(&seen);
    st->dx = 0.0; st->iter = 0;
    return st;
}

void orx_destroy(orx_state *st) {
    if (!st) return;
    dmap_free(&st->map);
    free(st->key); free(st->C); free(st->B); free(st->cand);
    free(st);
}

static double orx_gnorm_inf(const orx_state *st, int64_t k, const double *S, double *G) {
    const int k1 = st->k1;
    double m = 0.0;
    for (int a = 0; a < k1; a++) {
        double s = 0.0;
        for (int b = 0; b < k1; b++) s += st->C[k * k1 + b] * S[b * k1 + a];
        G[a] = 4.0 * st->B[k * k1 + a] + 4.0 * s;
        if (fabs(G[a]) > m) m = fabs(G[a]);
    }
    return m;
}

/* one iteration of Algorithm 3 */
static int orx_step1(orx_state *st) {
    const int k1 = st->k1;
    double S[XK_MAX * XK_MAX], G[XK_MAX], g[XK_MAX];
    for (int a = 0; a < k1 * k1; a++) S[a] = (double)st->S[a];
    int64_t best = -1;
    double gbest = -1.0;
    for (int64_t t = 0; t < st->ncand; t++) {
        int64_t k = st->cand[t];
        double gk = orx_gnorm_inf(st, k, S, G);
        if (best < 0 || gk > gbest || (gk == gbest && det_less(st->key[k], st->key[best]))) {
            best = k; gbest = gk;
            for (int a = 0; a < k1; a++) g[a] = G[a];
        }
    }
    if (best < 0) return -3;
    det_t Di = st->key[best];
    double c[XK_MAX];
    for (int a = 0; a < k1; a++) c[a] = st->C[best * k1 + a];
    double Hii = diag_sc(st->N, st->h, st->g, Di);
    double w[5];
    orx_quartic(k1, c, g, S, Hii, w);
    double eta = 0.0;
    if (w[4] > 0.0) eta = orc_line_search(w[1] / w[4], w[2] / w[4], w[3] / w[4]);
    st->ncand = 0;
    dmap seen;
    if (dmap_init(&seen, 1024)) return -1;
    int r = orx_row_step(st, Di, eta, g, &seen);
    dmap_free(&seen);
    if (r) return -1;
    double gn = 0.0;
    for (int a = 0; a < k1; a++) gn += g[a] * g[a];
    st->dx = st->theta * st->dx + (1.0 - st->theta) * fabs(eta) * sqrt(gn);
    st->iter++;
    return 0;
}

int orx_step(orx_state *st, int64_t n) {
    for (int64_t t = 0; t < n; t++) {
        int r = orx_step1(st);
        if (r) return r;
    }
    return 0;
}

/* energies: the k1 eigenvalues of the pencil (M, S), ascending (S = L L^T, eig of L^-1 M L^-T) */
int orx_energies(const orx_state *st, double *E) {
    const int k1 = st->k1;
    double L[XK_MAX * XK_MAX] = {0}, A[XK_MAX * XK_MAX], T[XK_MAX * XK_MAX], V[XK_MAX * XK_MAX];
    for (int i = 0; i < k1; i++)
        for (int j = 0; j <= i; j++) {
            double s = (double)st->S[i * k1 + j];
            for (int k = 0; k < j; k++) s -= L[i * k1 + k] * L[j * k1 + k];
            if (i == j) {
                if (!(s > 0.0)) return -1;
                L[i * k1 + i] = sqrt(s);
            } else {
                L[i * k1 + j] = s / L[j * k1 + j];
            }
        }
    /* T = L^-1 M (forward substitution per column), A = T L^-T */
    for (int col = 0; col < k1; col++)
        for (int i = 0; i < k1; i++) {
            double s = (double)st->M[i * k1 + col];
            for (int k = 0; k < i; k++) s -= L[i * k1 + k] * T[k * k1 + col];
            T[i * k1 + col] = s / L[i * k1 + i];
        }
    for (int row = 0; row < k1; row++)
        for (int i = 0; i < k1; i++) {
            double s = T[row * k1 + i];
            for (int k = 0; k < i; k++) s -= L[i * k1 + k] * A[row * k1 + k];
            A[row * k1 + i] = s / L[i * k1 + i];
        }
    for (int i = 0; i < k1; i++)
        for (int j = 0; j < i; j++) {
            double s = 0.5 * (A[i * k1 + j] + A[j * k1 + i]);
            A[i * k1 + j] = s; A[j * k1 + i] = s;
        }
    jacobi_eig(k1, A, E, V);
    for (int i = 0; i < k1; i++)
        for (int j = i + 1; j < k1; j++)
            if (E[j] < E[i]) { double t = E[i]; E[i] = E[j]; E[j] = t; }
    return 0;
}

/* S, M (as doubles, k1 x k1 each), dx, iterations, entries, elements, applied, dropped */
void orx_info(const orx_state *st, double *S, double *M, double *out) {
    const int k1 = st->k1;
    for (int a = 0; a < k1 * k1; a++) { S[a] = (double)st->S[a]; M[a] = (double)st->M[a]; }
    out[0] = st->dx; out[1] = (double)st->iter; out[2] = (double)st->n;
    out[3] = (double)st->elements; out[4] = (double)st->applied; out[5] = (double)st->dropped;
}

int64_t orx_export(const orx_state *st, uint64_t *keys, double *C, double *B, int64_t cap) {
    const int k1 = st->k1;
    int64_t n = st->n < cap ? st->n : cap;
    for (int64_t k = 0; k < n; k++) {
        keys[2 * k] = st->key[k].a; keys[2 * k + 1] = st->key[k].b;
        for (int a = 0; a < k1; a++) { C[k * k1 + a] = st->C[k * k1 + a]; B[k * k1 + a] = st->B[k * k1 + a]; }
    }
    return st->n;
}

void orx_last_step(const orx_state *st, uint64_t *key, double *eta) {
    key[0] = st->last_key.a; key[1] = st->last_key.b; *eta = st->last_eta;
}
