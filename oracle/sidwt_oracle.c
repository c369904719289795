/*
 * sidwt_oracle.c -- plain FP64 CPU oracle for multiresolution correlation of
 * complex signals in the shift-invariant DWT (SIDWT) domain by lifting
 * (Bhattacharya & Mahapatra, "A Novel Application of Lifting Scheme for
 * Multiresolution Correlation of Complex Radar Signals").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the CUDA
 * library.  It shares no code, header, table or constant generator with the
 * GPU path, and the GPU path never calls it.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it.
 *
 * Everything here is slow on purpose: straight loops over the definitions,
 * periodic indexing through a modulo helper, one lifting step at a time in the
 * order the factorisations print them.  Real lifting steps act on the real and
 * imaginary parts separately (Sec. IV, eq. 19; the global factor 2 of eq. 19
 * moves no peak and is dropped).
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *  - z^k acting on a phase sequence is an advance: (z^k s)[n] = s[n+k];
 *    a factor such as (1+z) therefore reads s[n]+s[n+1].  Lifting matrices
 *    are applied right to left.
 *  - Polyphase phases: e[n] = v[2n]; o[n] = v[2n+1] for LeGall 5/3 and
 *    CDF 9/7 (Sec. III-A, eq. 8-10).  For the causal Daubechies-4 form of
 *    eq. 17 the odd phase is o[n] = v[2n-1]: only that pairing reproduces the
 *    causal analysis polynomials printed in Sec. III-B.
 *  - Every signal is periodic (circular) at every level.
 *  - Lag convention: r_j[D] correlates the received y with the stored x
 *    delayed circularly by D, conj on the stored side, D in [0, L).
 *  - Scales j = 0..J.  For j < J the paper's form uses the level-(j+1)
 *    approximation and detail bands (eq. 5, 20); scale J uses the level-J
 *    approximations only (eq. 20a).
 *  - Integer 5/3 (only cited by the paper, Sec. I and V-B): floor-rounded
 *    reversible steps with the diagonal scalings dropped; x side
 *    o' = o - floor((e[n]+e[n+1])/2), e' = e + floor((o'[n-1]+o'[n]+2)/4);
 *    y side e' = e + floor((o[n]+o[n-1]+1)/2), o' = o - floor((e'[n]+e'[n+1]+2)/4).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_D4 0
#define OR_LEGALL53 1
#define OR_CDF97 2
#define OR_LEGALL53_INT 3
#define OR_CDF97_INT 4

#define OR_SIDE_X 0 /* stored (matching) signal: primal analysis P~(z^-1) */
#define OR_SIDE_Y 1 /* received signal: dual analysis P^T(z^-1)          */

static long wrap(long i, long m) {
    long r = i % m;
    return r < 0 ? r + m : r;
}

/* floor(a / b) for b > 0, written out so that it does not depend on how C
 * rounds a negative quotient. */
static int64_t floordiv(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return q;
}

/* ------------------------------------------------------------------------ */
/* Lifting constants.                                                        */
/* ------------------------------------------------------------------------ */

/* CDF 9/7 lifting parameters a, b, g, d and the scale x.  By default the
 * rational values of Table I (t = 5/4); oracle_set_cdf97_t selects another
 * member of the family of Sec. III-C Case II:
 *   a = (1 - 2t) / (4 (t - 1)), b = -(t - 1)^2, g = 1 / (4 t (t - 1)),
 *   d = t^3 - (7/4) t^2 + t, x = sqrt(2) / t.                                */
static double g97[5] = {-3.0 / 2.0, -1.0 / 16.0, 4.0 / 5.0, 15.0 / 32.0, 0.0};
static int g97_table = 1;
#define L97_A (g97[0])
#define L97_B (g97[1])
#define L97_G (g97[2])
#define L97_D (g97[3])
static double l97_x(void) { return g97_table ? 4.0 * sqrt(2.0) / 5.0 : g97[4]; }

/* t = 0 restores Table I; -1 for t = 1 (where a and g are undefined). */
int oracle_set_cdf97_t(double t) {
    if (t == 0.0) {
        g97[0] = -3.0 / 2.0;
        g97[1] = -1.0 / 16.0;
        g97[2] = 4.0 / 5.0;
        g97[3] = 15.0 / 32.0;
        g97_table = 1;
        return 0;
    }
    if (fabs(t - 1.0) < 1e-9 || t == 0.0) return -1;
    g97[0] = (1.0 - 2.0 * t) / (4.0 * (t - 1.0));
    g97[1] = -(t - 1.0) * (t - 1.0);
    g97[2] = 1.0 / (4.0 * t * (t - 1.0));
    g97[3] = t * t * t - 1.75 * t * t + t;
    g97[4] = sqrt(2.0) / t;
    g97_table = 0;
    return 0;
}

/* Exposed so that a test can compare them with the t-formulas of Sec. III-C. */
void oracle_cdf97_constants(double out[5]) {
    out[0] = L97_A;
    out[1] = L97_B;
    out[2] = L97_G;
    out[3] = L97_D;
    out[4] = l97_x();
}

/* ------------------------------------------------------------------------ */
/* One analysis level of a real periodic vector by lifting.                  */
/* ------------------------------------------------------------------------ */

static void split_phases(int filter, const double *v, long K, double *e, double *o) {
    long H = K / 2;
    for (long n = 0; n < H; ++n) {
        e[n] = v[2 * n];
        o[n] = (filter == OR_D4) ? v[wrap(2 * n - 1, K)] : v[2 * n + 1];
    }
}

/* Causal Daubechies-4, eq. 17, used on both sides (Sec. III-B, last
 * paragraph: the dual bases coincide for an orthogonal filterbank).
 * Right to left: predict o1 = o - sqrt3 e; update e1 = e + (sqrt3/4) o1 +
 * ((sqrt3-2)/4) z^-1 o1; the factor [1 0; 1 z^-1] gives o2 = e1 + z^-1 o1;
 * then diag((sqrt3+1)/sqrt2, (sqrt3-1)/sqrt2). */
static void lift_d4(const double *e, const double *o, long H, double *a, double *b) {
    const double s3 = sqrt(3.0), s2 = sqrt(2.0);
    const double k_lo = (s3 + 1.0) / s2, k_hi = (s3 - 1.0) / s2;
    double *o1 = malloc(sizeof(double) * H), *e1 = malloc(sizeof(double) * H);
    for (long n = 0; n < H; ++n) o1[n] = o[n] - s3 * e[n];
    for (long n = 0; n < H; ++n)
        e1[n] = e[n] + (s3 / 4.0) * o1[n] + ((s3 - 2.0) / 4.0) * o1[wrap(n - 1, H)];
    for (long n = 0; n < H; ++n) {
        double o2 = e1[n] + o1[wrap(n - 1, H)];
        a[n] = k_lo * e1[n];
        b[n] = k_hi * o2;
    }
    free(o1);
    free(e1);
}

/* LeGall 5/3 primal analysis (x side), Sec. III-C Case I:
 * P~(z^-1) = diag(1, 1/2) [1 (1+z^-1)/4; 0 1] [1 0; -(1+z)/2 1]. */
static void lift_53_x(const double *e, const double *o, long H, double *a, double *b) {
    double *o1 = malloc(sizeof(double) * H);
    for (long n = 0; n < H; ++n) o1[n] = o[n] - 0.5 * (e[n] + e[wrap(n + 1, H)]);
    for (long n = 0; n < H; ++n) {
        a[n] = e[n] + 0.25 * (o1[n] + o1[wrap(n - 1, H)]);
        b[n] = 0.5 * o1[n];
    }
    free(o1);
}

/* LeGall 5/3 dual analysis (y side), Sec. III-C Case I:
 * P^T(z^-1) = diag(1, 2) [1 0; -(1+z)/4 1] [1 (1+z^-1)/2; 0 1]. */
static void lift_53_y(const double *e, const double *o, long H, double *c, double *d) {
    double *e1 = malloc(sizeof(double) * H);
    for (long n = 0; n < H; ++n) e1[n] = e[n] + 0.5 * (o[n] + o[wrap(n - 1, H)]);
    for (long n = 0; n < H; ++n) {
        c[n] = e1[n];
        d[n] = 2.0 * (o[n] - 0.25 * (e1[n] + e1[wrap(n + 1, H)]));
    }
    free(e1);
}

/* CDF 9/7 primal analysis (x side), Sec. III-C Case II, with Table I:
 * P~(z^-1) = diag(x, 1/x) [1 d(1+z^-1); 0 1] [1 0; g(1+z) 1]
 *            [1 b(1+z^-1); 0 1] [1 0; a(1+z) 1]. */
static void lift_97_x(const double *e, const double *o, long H, double *a_out, double *b_out) {
    double *o1 = malloc(sizeof(double) * H), *e1 = malloc(sizeof(double) * H);
    double *o2 = malloc(sizeof(double) * H);
    const double x = l97_x();
    for (long n = 0; n < H; ++n) o1[n] = o[n] + L97_A * (e[n] + e[wrap(n + 1, H)]);
    for (long n = 0; n < H; ++n) e1[n] = e[n] + L97_B * (o1[n] + o1[wrap(n - 1, H)]);
    for (long n = 0; n < H; ++n) o2[n] = o1[n] + L97_G * (e1[n] + e1[wrap(n + 1, H)]);
    for (long n = 0; n < H; ++n) {
        double e2 = e1[n] + L97_D * (o2[n] + o2[wrap(n - 1, H)]);
        a_out[n] = x * e2;
        b_out[n] = o2[n] / x;
    }
    free(o1);
    free(e1);
    free(o2);
}

/* CDF 9/7 dual analysis (y side), Sec. III-C Case II:
 * P^T(z^-1) = diag(1/x, x) [1 0; -d(1+z) 1] [1 -g(1+z^-1); 0 1]
 *             [1 0; -b(1+z) 1] [1 -a(1+z^-1); 0 1]. */
static void lift_97_y(const double *e, const double *o, long H, double *c, double *d_out) {
    double *e1 = malloc(sizeof(double) * H), *o1 = malloc(sizeof(double) * H);
    double *e2 = malloc(sizeof(double) * H);
    const double x = l97_x();
    for (long n = 0; n < H; ++n) e1[n] = e[n] - L97_A * (o[n] + o[wrap(n - 1, H)]);
    for (long n = 0; n < H; ++n) o1[n] = o[n] - L97_B * (e1[n] + e1[wrap(n + 1, H)]);
    for (long n = 0; n < H; ++n) e2[n] = e1[n] - L97_G * (o1[n] + o1[wrap(n - 1, H)]);
    for (long n = 0; n < H; ++n) {
        double o2 = o1[n] - L97_D * (e2[n] + e2[wrap(n + 1, H)]);
        c[n] = e2[n] / x;
        d_out[n] = x * o2;
    }
    free(e1);
    free(o1);
    free(e2);
}

/* One analysis level of a real periodic vector v (length K, even) for the
 * floating-point filters.  side = OR_SIDE_X (primal) or OR_SIDE_Y (dual).
 * Writes the approximation a[K/2] and the detail b[K/2].  Returns 0, or -1
 * for an unsupported filter or an odd length. */
int oracle_lift_level(int filter, int side, const double *v, long K, double *a, double *b) {
    if (K < 2 || (K & 1)) return -1;
    long H = K / 2;
    double *e = malloc(sizeof(double) * H), *o = malloc(sizeof(double) * H);
    split_phases(filter, v, K, e, o);
    int rc = 0;
    switch (filter) {
    case OR_D4: lift_d4(e, o, H, a, b); break;
    case OR_LEGALL53:
        if (side == OR_SIDE_X) lift_53_x(e, o, H, a, b);
        else lift_53_y(e, o, H, a, b);
        break;
    case OR_CDF97:
        if (side == OR_SIDE_X) lift_97_x(e, o, H, a, b);
        else lift_97_y(e, o, H, a, b);
        break;
    default: rc = -1;
    }
    free(e);
    free(o);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Inverse lifting: each step of the forward factorisation undone in         */
/* reverse order (used for the perfect-reconstruction checks of eq. 11/13,   */
/* the causal D4 synthesis of Sec. III-B and Case I's scaled P(z)).          */
/* ------------------------------------------------------------------------ */

static void merge_phases(int filter, const double *e, const double *o, long K, double *v) {
    long H = K / 2;
    for (long n = 0; n < H; ++n) {
        v[2 * n] = e[n];
        if (filter == OR_D4) v[wrap(2 * n - 1, K)] = o[n];
        else v[2 * n + 1] = o[n];
    }
}

int oracle_lift_level_inv(int filter, int side, const double *a, const double *b, long K, double *v) {
    if (K < 2 || (K & 1)) return -1;
    long H = K / 2;
    double *e = malloc(sizeof(double) * H), *o = malloc(sizeof(double) * H);
    double *t1 = malloc(sizeof(double) * H), *t2 = malloc(sizeof(double) * H);
    int rc = 0;
    if (filter == OR_D4) {
        const double s3 = sqrt(3.0), s2 = sqrt(2.0);
        const double k_lo = (s3 + 1.0) / s2, k_hi = (s3 - 1.0) / s2;
        /* e1 = a/k_lo; o2 = b/k_hi; o1[n-1] = o2[n] - e1[n] */
        for (long n = 0; n < H; ++n) t1[n] = a[n] / k_lo;                       /* e1 */
        for (long n = 0; n < H; ++n) t2[wrap(n - 1, H)] = b[n] / k_hi - t1[n];  /* o1 */
        for (long n = 0; n < H; ++n)
            e[n] = t1[n] - (s3 / 4.0) * t2[n] - ((s3 - 2.0) / 4.0) * t2[wrap(n - 1, H)];
        for (long n = 0; n < H; ++n) o[n] = t2[n] + s3 * e[n];
    } else if (filter == OR_LEGALL53 && side == OR_SIDE_X) {
        for (long n = 0; n < H; ++n) t1[n] = 2.0 * b[n]; /* o1 */
        for (long n = 0; n < H; ++n) e[n] = a[n] - 0.25 * (t1[n] + t1[wrap(n - 1, H)]);
        for (long n = 0; n < H; ++n) o[n] = t1[n] + 0.5 * (e[n] + e[wrap(n + 1, H)]);
    } else if (filter == OR_LEGALL53 && side == OR_SIDE_Y) {
        for (long n = 0; n < H; ++n) t1[n] = 0.5 * b[n]; /* o1 */
        for (long n = 0; n < H; ++n) o[n] = t1[n] + 0.25 * (a[n] + a[wrap(n + 1, H)]);
        for (long n = 0; n < H; ++n) e[n] = a[n] - 0.5 * (o[n] + o[wrap(n - 1, H)]);
    } else if (filter == OR_CDF97 && side == OR_SIDE_X) {
        const double x = l97_x();
        double *o2 = malloc(sizeof(double) * H);
        for (long n = 0; n < H; ++n) o2[n] = b[n] * x;
        for (long n = 0; n < H; ++n) t1[n] = a[n] / x - L97_D * (o2[n] + o2[wrap(n - 1, H)]); /* e1 */
        for (long n = 0; n < H; ++n) t2[n] = o2[n] - L97_G * (t1[n] + t1[wrap(n + 1, H)]);     /* o1 */
        for (long n = 0; n < H; ++n) e[n] = t1[n] - L97_B * (t2[n] + t2[wrap(n - 1, H)]);
        for (long n = 0; n < H; ++n) o[n] = t2[n] - L97_A * (e[n] + e[wrap(n + 1, H)]);
        free(o2);
    } else if (filter == OR_CDF97 && side == OR_SIDE_Y) {
        const double x = l97_x();
        double *e2 = malloc(sizeof(double) * H);
        for (long n = 0; n < H; ++n) e2[n] = a[n] * x;
        for (long n = 0; n < H; ++n) t2[n] = b[n] / x + L97_D * (e2[n] + e2[wrap(n + 1, H)]); /* o1 */
        for (long n = 0; n < H; ++n) t1[n] = e2[n] + L97_G * (t2[n] + t2[wrap(n - 1, H)]);    /* e1 */
        for (long n = 0; n < H; ++n) o[n] = t2[n] + L97_B * (t1[n] + t1[wrap(n + 1, H)]);
        for (long n = 0; n < H; ++n) e[n] = t1[n] + L97_A * (o[n] + o[wrap(n - 1, H)]);
        free(e2);
    } else {
        rc = -1;
    }
    if (rc == 0) merge_phases(filter, e, o, K, v);
    free(e);
    free(o);
    free(t1);
    free(t2);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Mallat convolution-and-downsample filterbank (Sec. II, eq. 2 and the      */
/* recursion of [8] quoted in Sec. II): a[n] = sum_m lo[m] v[2n + off_lo[m]], */
/* b[n] = sum_m hi[m] v[2n + off_hi[m]], periodic.  The taps are supplied by  */
/* the caller (the printed filters of Sec. III), so this routine holds no     */
/* filter knowledge of its own.                                               */
/* ------------------------------------------------------------------------ */
void oracle_mallat_level(const double *v, long K, int n_lo, const int *off_lo, const double *lo,
                         int n_hi, const int *off_hi, const double *hi, double *a, double *b) {
    long H = K / 2;
    for (long n = 0; n < H; ++n) {
        double s = 0.0, t = 0.0;
        for (int m = 0; m < n_lo; ++m) s += lo[m] * v[wrap(2 * n + off_lo[m], K)];
        for (int m = 0; m < n_hi; ++m) t += hi[m] * v[wrap(2 * n + off_hi[m], K)];
        a[n] = s;
        b[n] = t;
    }
}

/* ------------------------------------------------------------------------ */
/* Reversible integer LeGall 5/3 (Sec. I and V-B, via ref. [25]).            */
/* ------------------------------------------------------------------------ */
int oracle_int53_level(int side, const int64_t *v, long K, int64_t *a, int64_t *b) {
    if (K < 2 || (K & 1)) return -1;
    long H = K / 2;
    int64_t *e = malloc(sizeof(int64_t) * H), *o = malloc(sizeof(int64_t) * H);
    int64_t *t = malloc(sizeof(int64_t) * H);
    for (long n = 0; n < H; ++n) {
        e[n] = v[2 * n];
        o[n] = v[2 * n + 1];
    }
    if (side == OR_SIDE_X) {
        for (long n = 0; n < H; ++n) t[n] = o[n] - floordiv(e[n] + e[wrap(n + 1, H)], 2);
        for (long n = 0; n < H; ++n) {
            a[n] = e[n] + floordiv(t[wrap(n - 1, H)] + t[n] + 2, 4);
            b[n] = t[n];
        }
    } else {
        for (long n = 0; n < H; ++n) t[n] = e[n] + floordiv(o[n] + o[wrap(n - 1, H)] + 1, 2);
        for (long n = 0; n < H; ++n) {
            a[n] = t[n];
            b[n] = o[n] - floordiv(t[n] + t[wrap(n + 1, H)] + 2, 4);
        }
    }
    free(e);
    free(o);
    free(t);
    return 0;
}

int oracle_int53_level_inv(int side, const int64_t *a, const int64_t *b, long K, int64_t *v) {
    if (K < 2 || (K & 1)) return -1;
    long H = K / 2;
    int64_t *e = malloc(sizeof(int64_t) * H), *o = malloc(sizeof(int64_t) * H);
    if (side == OR_SIDE_X) {
        for (long n = 0; n < H; ++n) e[n] = a[n] - floordiv(b[wrap(n - 1, H)] + b[n] + 2, 4);
        for (long n = 0; n < H; ++n) o[n] = b[n] + floordiv(e[n] + e[wrap(n + 1, H)], 2);
    } else {
        for (long n = 0; n < H; ++n) o[n] = b[n] + floordiv(a[n] + a[wrap(n + 1, H)] + 2, 4);
        for (long n = 0; n < H; ++n) e[n] = a[n] - floordiv(o[n] + o[wrap(n - 1, H)] + 1, 2);
    }
    for (long n = 0; n < H; ++n) {
        v[2 * n] = e[n];
        v[2 * n + 1] = o[n];
    }
    free(e);
    free(o);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Reversible integer CDF 9/7: the steps of Table I with dyadic constants     */
/* (a = -3/2, b = -1/16, g = 205/256 ~ 4/5, d = 15/32), each update rounded   */
/* to the nearest integer (floor(c s + 1/2)), the diagonal scalings dropped   */
/* (x on one side, 1/x on the other: they cancel in the pairing).            */
/* x side (P~): o += R(a (e[n] + e[n+1])); e += R(b (o[n] + o[n-1]));       */
/*              o += R(g (e[n] + e[n+1])); e += R(d (o[n] + o[n-1])).        */
/* y side (P^T): e -= R(a (o[n] + o[n-1])); o -= R(b (e[n] + e[n+1]));      */
/*              e -= R(g (o[n] + o[n-1])); o -= R(d (e[n] + e[n+1])).        */
/* ------------------------------------------------------------------------ */
static const int64_t I97_K[4] = {-3, -1, 205, 15}; /* numerators of a, b, g, d */
static const int I97_M[4] = {1, 4, 8, 5};          /* denominators 2^m          */

/* R(k s / 2^m) = floor((k s + 2^(m-1)) / 2^m) */
static int64_t rdy(int64_t k, int m, int64_t s) { return floordiv(k * s + ((int64_t)1 << (m - 1)), (int64_t)1 << m); }

int oracle_int97_level(int side, const int64_t *v, long K, int64_t *a, int64_t *b) {
    if (K < 2 || (K & 1)) return -1;
    long H = K / 2;
    int64_t *e = malloc(sizeof(int64_t) * H), *o = malloc(sizeof(int64_t) * H);
    for (long n = 0; n < H; ++n) {
        e[n] = v[2 * n];
        o[n] = v[2 * n + 1];
    }
    for (int s = 0; s < 4; ++s) {
        const int odd_target = (side == OR_SIDE_X) ? (s % 2 == 0) : (s % 2 == 1);
        const int64_t k = (side == OR_SIDE_X) ? I97_K[s] : -I97_K[s];
        if (odd_target) { /* o[n] += R(c (e[n] + e[n+1])) */
            for (long n = 0; n < H; ++n) o[n] += rdy(k, I97_M[s], e[n] + e[wrap(n + 1, H)]);
        } else { /* e[n] += R(c (o[n] + o[n-1])) */
            for (long n = 0; n < H; ++n) e[n] += rdy(k, I97_M[s], o[n] + o[wrap(n - 1, H)]);
        }
    }
    for (long n = 0; n < H; ++n) {
        a[n] = e[n];
        b[n] = o[n];
    }
    free(e);
    free(o);
    return 0;
}

int oracle_int97_level_inv(int side, const int64_t *a, const int64_t *b, long K, int64_t *v) {
    if (K < 2 || (K & 1)) return -1;
    long H = K / 2;
    int64_t *e = malloc(sizeof(int64_t) * H), *o = malloc(sizeof(int64_t) * H);
    for (long n = 0; n < H; ++n) {
        e[n] = a[n];
        o[n] = b[n];
    }
    for (int s = 3; s >= 0; --s) {
        const int odd_target = (side == OR_SIDE_X) ? (s % 2 == 0) : (s % 2 == 1);
        const int64_t k = (side == OR_SIDE_X) ? I97_K[s] : -I97_K[s];
        if (odd_target) {
            for (long n = 0; n < H; ++n) o[n] -= rdy(k, I97_M[s], e[n] + e[wrap(n + 1, H)]);
        } else {
            for (long n = 0; n < H; ++n) e[n] -= rdy(k, I97_M[s], o[n] + o[wrap(n - 1, H)]);
        }
    }
    for (long n = 0; n < H; ++n) {
        v[2 * n] = e[n];
        v[2 * n + 1] = o[n];
    }
    free(e);
    free(o);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Complex helpers: real transforms on Re and Im separately (eq. 19).        */
/* Complex vectors are interleaved (re, im) doubles.                          */
/* ------------------------------------------------------------------------ */

static int level_complex(int filter, int side, const double *v, long K, double *a, double *b) {
    long H = K / 2;
    double *pr = malloc(sizeof(double) * K), *pi = malloc(sizeof(double) * K);
    double *ar = malloc(sizeof(double) * H), *ai = malloc(sizeof(double) * H);
    double *br = malloc(sizeof(double) * H), *bi = malloc(sizeof(double) * H);
    for (long k = 0; k < K; ++k) {
        pr[k] = v[2 * k];
        pi[k] = v[2 * k + 1];
    }
    int rc = 0;
    if (filter == OR_LEGALL53_INT || filter == OR_CDF97_INT) {
        int64_t *iv = malloc(sizeof(int64_t) * K), *ia = malloc(sizeof(int64_t) * H),
                *ib = malloc(sizeof(int64_t) * H);
        for (int part = 0; part < 2; ++part) {
            double *src = part ? pi : pr;
            for (long k = 0; k < K; ++k) iv[k] = (int64_t)llround(src[k]);
            if (filter == OR_CDF97_INT)
                oracle_int97_level(side, iv, K, ia, ib);
            else
                oracle_int53_level(side, iv, K, ia, ib);
            for (long n = 0; n < H; ++n) {
                (part ? ai : ar)[n] = (double)ia[n];
                (part ? bi : br)[n] = (double)ib[n];
            }
        }
        free(iv);
        free(ia);
        free(ib);
    } else {
        rc |= oracle_lift_level(filter, side, pr, K, ar, br);
        rc |= oracle_lift_level(filter, side, pi, K, ai, bi);
    }
    for (long n = 0; n < H; ++n) {
        a[2 * n] = ar[n];
        a[2 * n + 1] = ai[n];
        b[2 * n] = br[n];
        b[2 * n + 1] = bi[n];
    }
    free(pr);
    free(pi);
    free(ar);
    free(ai);
    free(br);
    free(bi);
    return rc;
}

/* Circular delay of a complex vector: out[n] = v[(n - D) mod K]. */
static void delay_complex(const double *v, long K, long D, double *out) {
    for (long n = 0; n < K; ++n) {
        long s = wrap(n - D, K);
        out[2 * n] = v[2 * s];
        out[2 * n + 1] = v[2 * s + 1];
    }
}

static int check_shape(int filter, long N, int J) {
    if (filter < 0 || filter > 4) return -1;
    if (J < 1 || J > 30 || N < 2) return -1;
    if (N % (1L << J) != 0) return -1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Received-signal pyramid: J levels of dual analysis of y (Sec. III-C,      */
/* Fig. 3(b)/4(b); D4 uses eq. 17 on both sides).  Output layout, complex:    */
/* level j = 1..J at offset 2N - 4*(N >> j): c_j[N >> j] then d_j[N >> j].    */
/* energies (optional) gets ||c_j||^2 for j = 0..J (c_0 = y), eq. 1.          */
/* Integer 5/3 inputs are integral doubles and outputs are exact integers.    */
/* ------------------------------------------------------------------------ */
int oracle_pyramid_y(int filter, const double *y, long N, int J, double *out, double *energies) {
    if (check_shape(filter, N, J)) return -1;
    double *cur = malloc(sizeof(double) * 2 * N);
    memcpy(cur, y, sizeof(double) * 2 * N);
    if (energies) {
        double s = 0.0;
        for (long k = 0; k < N; ++k) s += cur[2 * k] * cur[2 * k] + cur[2 * k + 1] * cur[2 * k + 1];
        energies[0] = s;
    }
    long K = N;
    for (int j = 1; j <= J; ++j) {
        long H = K / 2;
        double *c = out + 2 * (2 * N - 4 * (N >> j));
        double *d = c + 2 * H;
        if (level_complex(filter, OR_SIDE_Y, cur, K, c, d)) {
            free(cur);
            return -1;
        }
        memcpy(cur, c, sizeof(double) * 2 * H);
        if (energies) {
            double s = 0.0;
            for (long k = 0; k < H; ++k) s += c[2 * k] * c[2 * k] + c[2 * k + 1] * c[2 * k + 1];
            energies[j] = s;
        }
        K = H;
    }
    free(cur);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* SIDWT tree of the stored signal x (Sec. II, Fig. 1 and 5; eq. 5).         */
/* Level j variant r (0 <= r < 2^j) is the level-j analysis of x delayed by  */
/* r.  From level j to j+1 the even child of variant r is the analysis of    */
/* variant r itself; the odd child is the analysis of variant r delayed by   */
/* one level-j sample, which is variant r + 2^j (a delay of 2^j at level 0). */
/* Output layout, complex: level j = 1..J at offset 2N(j-1):                 */
/*   A[2^j][N >> j] (approximations) then B[2^j][N >> j] (details).          */
/* energies (optional): for j = 0..J, 2^j values ||X_{j,r}||^2 at offset      */
/* 2^j - 1 (X_{0,0} = x).                                                     */
/* ------------------------------------------------------------------------ */
int oracle_tree_x(int filter, const double *x, long N, int J, double *out, double *energies) {
    if (check_shape(filter, N, J)) return -1;
    /* prev holds the 2^j level-j approximation variants, each N>>j complex. */
    double *prev = malloc(sizeof(double) * 2 * N);
    double *next = malloc(sizeof(double) * 2 * N);
    double *tmp = malloc(sizeof(double) * 2 * N);
    memcpy(prev, x, sizeof(double) * 2 * N);
    if (energies) {
        double s = 0.0;
        for (long k = 0; k < N; ++k) s += x[2 * k] * x[2 * k] + x[2 * k + 1] * x[2 * k + 1];
        energies[0] = s;
    }
    for (int j = 0; j < J; ++j) {
        long K = N >> j, H = K / 2, nv = 1L << j;
        double *A = out + 2 * (2 * N * (long)j);
        double *B = A + 2 * N;
        for (long r = 0; r < nv; ++r) {
            const double *X = prev + 2 * r * K;
            /* even child: variant r */
            if (level_complex(filter, OR_SIDE_X, X, K, A + 2 * r * H, B + 2 * r * H)) goto fail;
            /* odd child: variant r delayed by one level-j sample = variant r + 2^j */
            delay_complex(X, K, 1, tmp);
            if (level_complex(filter, OR_SIDE_X, tmp, K, A + 2 * (r + nv) * H, B + 2 * (r + nv) * H))
                goto fail;
        }
        memcpy(next, A, sizeof(double) * 2 * N);
        double *sw = prev;
        prev = next;
        next = sw;
        if (energies) {
            for (long r = 0; r < 2 * nv; ++r) {
                double s = 0.0;
                const double *X = prev + 2 * r * H;
                for (long k = 0; k < H; ++k) s += X[2 * k] * X[2 * k] + X[2 * k + 1] * X[2 * k + 1];
                energies[(2 * nv - 1) + r] = s;
            }
        }
    }
    free(prev);
    free(next);
    free(tmp);
    return 0;
fail:
    free(prev);
    free(next);
    free(tmp);
    return -1;
}

/* Level-j analysis of x delayed by D, computed the long way: delay x at level
 * 0, then run j levels of primal analysis (used to pin the shift-circulant
 * identity of Sec. II).  out: approximation (N>>j complex); det (optional):
 * the level-j detail (N>>j complex), for j >= 1. */
int oracle_delayed_analysis_x(int filter, const double *x, long N, int j, long D, double *out,
                              double *det) {
    if (filter < 0 || filter > 4 || j < 0 || N % (1L << j) != 0) return -1;
    double *cur = malloc(sizeof(double) * 2 * N);
    double *b = malloc(sizeof(double) * 2 * N);
    delay_complex(x, N, D, cur);
    long K = N;
    for (int l = 0; l < j; ++l) {
        double *a = malloc(sizeof(double) * K);
        if (level_complex(filter, OR_SIDE_X, cur, K, a, b)) {
            free(a);
            free(cur);
            free(b);
            return -1;
        }
        memcpy(cur, a, sizeof(double) * K);
        free(a);
        K /= 2;
    }
    memcpy(out, cur, sizeof(double) * 2 * K);
    if (det && j >= 1) memcpy(det, b, sizeof(double) * 2 * K);
    free(cur);
    free(b);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Correlation at every lag and every scale.                                 */
/* r has (J+1) rows of N complex values: r[j][D], D = 0..N-1.                */
/*                                                                           */
/* form 0 -- definition: r_j[D] = sum_k conj(X_{j,D}[k]) c_j[k], where        */
/*   X_{j,D} is the level-j approximation of x delayed by D (by the shift-    */
/*   circulant identity, variant D mod 2^j rolled by D div 2^j) and c_j the   */
/*   level-j approximation of y (X_0 = x, c_0 = y).                           */
/* form 1 -- the paper's DWT-domain form, eq. 5 / 20 for j < J:               */
/*   r_j[D] = <A_{j+1,D}, c_{j+1}> + <B_{j+1,D}, d_{j+1}> with variant        */
/*   D mod 2^{j+1} rolled by D div 2^{j+1}; eq. 20a for j = J (A only).       */
/* Both use <u, v> = sum conj(u) v.                                           */
/* ------------------------------------------------------------------------ */

static void cdot_roll(const double *u, const double *v, long K, long q, double *re, double *im) {
    /* sum_k conj(u[(k - q) mod K]) v[k] */
    double sr = 0.0, si = 0.0;
    for (long k = 0; k < K; ++k) {
        long s = wrap(k - q, K);
        double ur = u[2 * s], ui = u[2 * s + 1], vr = v[2 * k], vi = v[2 * k + 1];
        sr += ur * vr + ui * vi;
        si += ur * vi - ui * vr;
    }
    *re += sr;
    *im += si;
}

static int correlate_one(int filter, const double *x, const double *y, long N, int J, double *r,
                         int form) {
    size_t tree_len = (size_t)2 * N * J * 2; /* doubles */
    size_t pyr_len = (size_t)2 * (2 * N) * 2;
    double *tree = malloc(sizeof(double) * tree_len);
    double *pyr = malloc(sizeof(double) * pyr_len);
    if (oracle_tree_x(filter, x, N, J, tree, NULL) || oracle_pyramid_y(filter, y, N, J, pyr, NULL)) {
        free(tree);
        free(pyr);
        return -1;
    }
    for (int j = 0; j <= J; ++j) {
        double *rj = r + 2 * (size_t)N * j;
        if (form == 0) {
            long K = N >> j, nv = 1L << j;
            /* level-j approximations of x (variants) and y */
            const double *Xv = (j == 0) ? x : tree + 2 * (2 * N * (long)(j - 1));
            const double *cj = (j == 0) ? y : pyr + 2 * (2 * N - 4 * (N >> j));
            for (long D = 0; D < N; ++D) {
                long rr = D % nv, q = D / nv;
                double re = 0.0, im = 0.0;
                cdot_roll(Xv + 2 * rr * K, cj, K, q, &re, &im);
                rj[2 * D] = re;
                rj[2 * D + 1] = im;
            }
        } else {
            int lev = (j < J) ? j + 1 : J;
            long K = N >> lev, nv = 1L << lev;
            const double *Av = tree + 2 * (2 * N * (long)(lev - 1));
            const double *Bv = Av + 2 * N;
            const double *c = pyr + 2 * (2 * N - 4 * (N >> lev));
            const double *d = c + 2 * K;
            for (long D = 0; D < N; ++D) {
                long rr = D % nv, q = D / nv;
                double re = 0.0, im = 0.0;
                cdot_roll(Av + 2 * rr * K, c, K, q, &re, &im);
                if (j < J) cdot_roll(Bv + 2 * rr * K, d, K, q, &re, &im);
                rj[2 * D] = re;
                rj[2 * D + 1] = im;
            }
        }
    }
    free(tree);
    free(pyr);
    return 0;
}

int oracle_correlate(int filter, const double *x, const double *y, long N, int J, double *r, int form) {
    if (check_shape(filter, N, J) || form < 0 || form > 1) return -1;
    return correlate_one(filter, x, y, N, J, r, form);
}

/* Textbook circular cross-correlation in the sample domain:
 * r[D] = sum_n conj(x[(n - D) mod N]) y[n]. */
void oracle_brute_xcorr(const double *x, const double *y, long N, double *r) {
    for (long D = 0; D < N; ++D) {
        double re = 0.0, im = 0.0;
        cdot_roll(x, y, N, D, &re, &im);
        r[2 * D] = re;
        r[2 * D + 1] = im;
    }
}

/* Peak per scale: lag = argmax_D |r_j[D]| (first maximum in increasing D),
 * mag = |r_j[lag]|, norm = mag / sqrt(E_x[j][lag mod 2^j] * E_y[j]) with the
 * energies of eq. 1 (definition-form normalisation). */
static void peaks_from_r(const double *r, long N, int J, const double *ex, const double *ey,
                         int32_t *lag, double *mag, double *norm) {
    for (int j = 0; j <= J; ++j) {
        const double *rj = r + 2 * (size_t)N * j;
        long best = 0;
        double bv = -1.0;
        for (long D = 0; D < N; ++D) {
            double m2 = rj[2 * D] * rj[2 * D] + rj[2 * D + 1] * rj[2 * D + 1];
            if (m2 > bv) {
                bv = m2;
                best = D;
            }
        }
        lag[j] = (int32_t)best;
        mag[j] = sqrt(bv);
        long v = best % (1L << j);
        double den = sqrt(ex[(1L << j) - 1 + v] * ey[j]);
        norm[j] = den > 0.0 ? mag[j] / den : 0.0;
    }
}

/* Correlate a batch of pairs (x_p, y_p), each N complex, and return for every
 * pair and scale the peak lag, |r| at the peak and the normalised value.
 * r_out (optional) receives the full r[p][j][D].  Pairs run in parallel with
 * OpenMP when the library is built with it; nthreads <= 0 keeps the default.
 * Returns the number of threads used, or -1 on a bad shape. */
int oracle_correlate_batch(int filter, const double *x, const double *y, long P, long N, int J,
                           int form, int32_t *lag, double *mag, double *norm, double *r_out,
                           int nthreads) {
    if (check_shape(filter, N, J) || P < 0) return -1;
    int used = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#else
    (void)nthreads;
#endif
    int bad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
#endif
    for (long p = 0; p < P; ++p) {
        const double *xp = x + 2 * (size_t)N * p, *yp = y + 2 * (size_t)N * p;
        double *r = r_out ? r_out + 2 * (size_t)N * (J + 1) * p
                          : malloc(sizeof(double) * 2 * (size_t)N * (J + 1));
        double *tree = malloc(sizeof(double) * (size_t)4 * N * J);
        double *pyr = malloc(sizeof(double) * (size_t)4 * N);
        double *ex = malloc(sizeof(double) * ((size_t)2 << J));
        double *ey = malloc(sizeof(double) * (J + 1));
        if (correlate_one(filter, xp, yp, N, J, r, form) || oracle_tree_x(filter, xp, N, J, tree, ex) ||
            oracle_pyramid_y(filter, yp, N, J, pyr, ey)) {
            bad |= 1;
        } else {
            peaks_from_r(r, N, J, ex, ey, lag + (J + 1) * p, mag + (J + 1) * p, norm + (J + 1) * p);
        }
        if (!r_out) free(r);
        free(tree);
        free(pyr);
        free(ex);
        free(ey);
    }
    return bad ? -1 : used;
}

/* Batch of pairs of mixed shapes: pair i has filter f[i], length N[i] and
 * depth J[i]; x_i and y_i start at complex offset off[i] of the packed
 * arrays; its J[i]+1 peak records start at slot[i].  Pairs run in parallel
 * with OpenMP.  Returns the number of threads used, or -1 on a bad shape. */
int oracle_correlate_mixed(long P, const int *f, const long *N, const int *J, const long *off, const long *slot,
                           const double *x, const double *y, int32_t *lag, double *mag, double *norm,
                           int nthreads) {
    int used = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#else
    (void)nthreads;
#endif
    int bad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
#endif
    for (long i = 0; i < P; ++i) {
        long s = slot[i];
        if (oracle_correlate_batch(f[i], x + 2 * off[i], y + 2 * off[i], 1, N[i], J[i], 1, lag + s, mag + s,
                                   norm + s, NULL, 1) < 0)
            bad |= 1;
    }
    return bad ? -1 : used;
}
