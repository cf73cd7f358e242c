/*
 * oracle.c -- plain, slow, sequential CPU oracle for classical BiCGStab
 * (Algorithm 1, van der Vorst) and pipelined BiCGStab (Algorithm 2,
 * Cools-Vanroose) as stated in Section 2 of "Robustness and Accuracy in
 * Pipelined Bi-Conjugate Gradient Stabilized Method: A Comparative Study"
 * (Havdiak, Aliaga, Iakymchuk, arXiv 2404.13216), in IEEE-754 binary64 as the
 * experiments of Section 3 use.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  The GPU library shares no code,
 * header, table or constant with it.
 *
 * Dot products come in two modes:
 *   plain : s = +0; for i in index order: s = fma(a_i, b_i, s)
 *   exact : the real sum  sum_i a_i*b_i  is formed exactly in a big integer and
 *           rounded to nearest-even once.  This is the accuracy guarantee the
 *           paper takes from ExBLAS (long accumulator, Section 2); the oracle
 *           reaches it by a different route (integer mantissa products added
 *           into a sign-magnitude big integer scaled by 2^-2148).
 *
 * Readings of the paper that this file implements (the paper is silent or
 * garbled on each):
 *   R1  Algorithm 2's "w_0 := A - r_0" is read as w_0 := A r_0 (the invariant
 *       w_i = A r_i and t_0 := A w_0 in the next line fix it).
 *   R2  In both algorithms the symbol w_i names two things: the scalar
 *       (q_i,y_i)/(y_i,y_i) (called omega here) and the vector A r_i (called w).
 *   R3  The shadow residual is r_0; rho_i denotes (r_0, r_i).
 *   R4  Algorithm 2 at i = 0: beta_{-1} = 0, so p_0 = r_0, s_0 = w_0, z_0 = t_0
 *       (bit copies).
 *   R5  Fixed rounding forms (fma = one rounding):
 *         SpMV row      acc = +0; acc = fma(val_k, x[col_k], acc) in stored order
 *         r_0           b_i - (A x_0)_i
 *         p             fma(beta, fma(-omega, s_old, p_old), r)   (s, z alike)
 *         q, y          fma(-alpha, s, r),  fma(-alpha, z, w)
 *         x             fma(omega, q, fma(alpha, p, x))
 *         r             fma(-omega, y, q)
 *         w (Alg. 2)    fma(-omega, fma(-alpha, v, t), y)
 *         omega         qy / yy
 *         beta          (alpha / omega) * (rho_new / rho_old)
 *         alpha_{i+1}   rho_new / ((rw + beta*rs) - (beta*omega)*rz)
 *         alpha_i (A1)  rho_i / (r_0, s_i)
 *   R6  Stopping: res_k = sqrt((r_k,r_k)) / sqrt((b,b)) in the solve's dot mode
 *       (sqrt((b,b)) replaced by 1 when b = 0); tested at k = 0 and after each
 *       r_{i+1}.  When res_k <= target the true residual
 *       ||b - A x||_2 / ||b||_2 (fixed SpMV, exact dot) is formed; the solve
 *       stops if it is <= tol, else target := tol * (tol / true) and the
 *       iteration goes on unchanged.  iters counts completed loop bodies.
 *   R7  Breakdown: yy = 0 gives omega = 0; the x and r updates still run and the
 *       stop test is applied, then BREAKDOWN.  Non-finite beta or alpha, or
 *       rho_new = 0, give BREAKDOWN.  A non-finite dot gives NONFINITE.
 *   R8  Exact dot: exact zero gives +0; ties to even; subnormal results exact
 *       at 2^-1074; overflow gives +-inf; any non-finite operand gives NaN.
 *   R9  Residual replacement (the p-BiCGStabRR of Section 2, period k): at the
 *       start of every iteration i > 0 with i mod k = 0, r_i := b - A x_i,
 *       w_i := A r_i, p_i by its recurrence (with the new r_i),
 *       s_i := A p_i, z_i := A s_i, t_i := A w_i; the scalars are kept.  The
 *       paper gives no more detail; k = 0 is plain Algorithm 2.
 *   R10 Right Jacobi preconditioning (orc_solve_jacobi, M = diag(A)): the
 *       algorithms run on A M^-1 y = b and x = M^-1 y, with the forms given
 *       above that function.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_CONVERGED = 0, ORC_MAXIT = 1, ORC_BREAKDOWN = 2, ORC_NONFINITE = 3, ORC_INVALID = -1 };
enum { ORC_BICGSTAB = 0, ORC_PIPELINED = 1 };
enum { ORC_PLAIN = 0, ORC_EXACT = 1 };

/* ------------------------------------------------------------------------ */
/* Exact accumulator: value = (pos - neg) * 2^-ORC_SCALE, pos/neg magnitudes  */
/* in little-endian base-2^32 limbs.  Every exact product of two finite      */
/* doubles is an integer multiple of 2^-2148 below 2^2048, so 136 limbs      */
/* (4352 bits) hold any sum of fewer than 2^150 such products.               */
/* ------------------------------------------------------------------------ */
#define ORC_LIMBS 136
#define ORC_SCALE 2148

typedef struct {
    uint32_t pos[ORC_LIMBS];
    uint32_t neg[ORC_LIMBS];
    int nonfinite;
} orc_acc;

static void mag_add_at(uint32_t *m, int k, uint64_t v)
{
    /* m += v * 2^(32k), carries propagated upward */
    while (v != 0 && k < ORC_LIMBS) {
        uint64_t s = (uint64_t)m[k] + (v & 0xffffffffu);
        m[k] = (uint32_t)s;
        v = (v >> 32) + (s >> 32);
        k++;
    }
}

/* split a finite double into (sign, integer mantissa, exponent of its LSB) */
static void decode(double a, int *sign, uint64_t *mant, int *lsbexp)
{
    uint64_t bits;
    memcpy(&bits, &a, sizeof bits);
    *sign = (int)(bits >> 63);
    int e = (int)((bits >> 52) & 0x7ff);
    uint64_t f = bits & ((UINT64_C(1) << 52) - 1);
    if (e == 0) {            /* zero or subnormal: f * 2^-1074 */
        *mant = f;
        *lsbexp = -1074;
    } else {                 /* normal: (2^52 + f) * 2^(e-1075) */
        *mant = f | (UINT64_C(1) << 52);
        *lsbexp = e - 1075;
    }
}

static int is_finite_bits(double a)
{
    uint64_t bits;
    memcpy(&bits, &a, sizeof bits);
    return ((bits >> 52) & 0x7ff) != 0x7ff;
}

/* add the exact product a*b into the accumulator */
static void acc_add_product(orc_acc *acc, double a, double b)
{
    if (!is_finite_bits(a) || !is_finite_bits(b)) {
        acc->nonfinite = 1;
        return;
    }
    int sa, sb, ea, eb;
    uint64_t ma, mb;
    decode(a, &sa, &ma, &ea);
    decode(b, &sb, &mb, &eb);
    if (ma == 0 || mb == 0)
        return;
    unsigned __int128 prod = (unsigned __int128)ma * mb;   /* < 2^106, exact */
    int off = ea + eb + ORC_SCALE;                          /* bit offset, >= 0 */
    int k = off / 32, r = off % 32;
    uint32_t *m = (sa ^ sb) ? acc->neg : acc->pos;
    for (int j = 0; j < 4; j++) {
        uint64_t piece = (uint64_t)(prod >> (32 * j)) & 0xffffffffu;
        mag_add_at(m, k + j, piece << r);                   /* < 2^63 */
    }
}

static void acc_merge(orc_acc *dst, const orc_acc *src)
{
    for (int k = 0; k < ORC_LIMBS; k++) {
        mag_add_at(dst->pos, k, src->pos[k]);
        mag_add_at(dst->neg, k, src->neg[k]);
    }
    dst->nonfinite |= src->nonfinite;
}

/* compare magnitudes: -1, 0, +1 */
static int mag_cmp(const uint32_t *a, const uint32_t *b)
{
    for (int k = ORC_LIMBS - 1; k >= 0; k--) {
        if (a[k] != b[k])
            return a[k] < b[k] ? -1 : 1;
    }
    return 0;
}

/* d = a - b, requires a >= b */
static void mag_sub(uint32_t *d, const uint32_t *a, const uint32_t *b)
{
    int64_t borrow = 0;
    for (int k = 0; k < ORC_LIMBS; k++) {
        int64_t s = (int64_t)a[k] - (int64_t)b[k] - borrow;
        borrow = s < 0;
        d[k] = (uint32_t)(s + (borrow ? (INT64_C(1) << 32) : 0));
    }
}

static int mag_bit(const uint32_t *m, int i)
{
    return (int)((m[i / 32] >> (i % 32)) & 1u);
}

/* signed difference pos - neg as (sign, magnitude) */
static void acc_signed(const orc_acc *acc, int *neg_sign, uint32_t *mag)
{
    if (mag_cmp(acc->pos, acc->neg) >= 0) {
        *neg_sign = 0;
        mag_sub(mag, acc->pos, acc->neg);
    } else {
        *neg_sign = 1;
        mag_sub(mag, acc->neg, acc->pos);
    }
}

/* round (sign, magnitude * 2^-2148) to the nearest double, ties to even */
static double round_mag(int neg_sign, const uint32_t *mag)
{
    int h = -1;
    for (int i = ORC_LIMBS * 32 - 1; i >= 0; i--) {
        if (mag_bit(mag, i)) {
            h = i;
            break;
        }
    }
    if (h < 0)
        return 0.0;                                  /* exact zero is +0 */
    /* the kept bits are [lsb, h]; 1074 = position of 2^-1074 */
    int lsb = h - 52;
    if (lsb < 1074)
        lsb = 1074;
    uint64_t m = 0;
    for (int i = h; i >= lsb; i--)
        m = (m << 1) | (uint64_t)mag_bit(mag, i);
    int rbit = (lsb >= 1 && lsb - 1 <= h) ? mag_bit(mag, lsb - 1) : 0;
    int sticky = 0;
    for (int i = lsb - 2; i >= 0; i--) {
        if (mag_bit(mag, i)) {
            sticky = 1;
            break;
        }
    }
    if (rbit && (sticky || (m & 1u)))
        m += 1;                                       /* m <= 2^53, exact in double */
    double v = ldexp((double)m, lsb - ORC_SCALE);     /* exact or +inf on overflow */
    return neg_sign ? -v : v;
}

static double acc_round(const orc_acc *acc)
{
    if (acc->nonfinite)
        return NAN;
    uint32_t mag[ORC_LIMBS];
    int s;
    acc_signed(acc, &s, mag);
    return round_mag(s, mag);
}

/* ------------------------------------------------------------------------ */
/* dot products                                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
    const double *a, *b;
    int64_t lo, hi;
    orc_acc acc;
} dot_job;

static void *dot_worker(void *p)
{
    dot_job *j = (dot_job *)p;
    for (int64_t i = j->lo; i < j->hi; i++)
        acc_add_product(&j->acc, j->a[i], j->b[i]);
    return NULL;
}

static void exact_acc_into(orc_acc *out, int64_t n, const double *a, const double *b, int nthreads)
{
    memset(out, 0, sizeof *out);
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > 64)
        nthreads = 64;
    if (n < 65536)
        nthreads = 1;
    if (nthreads == 1) {
        for (int64_t i = 0; i < n; i++)
            acc_add_product(out, a[i], b[i]);
        return;
    }
    dot_job *jobs = (dot_job *)calloc((size_t)nthreads, sizeof(dot_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    int *started = (int *)calloc((size_t)nthreads, sizeof(int));
    for (int t = 0; t < nthreads; t++) {
        jobs[t].a = a;
        jobs[t].b = b;
        jobs[t].lo = n * t / nthreads;
        jobs[t].hi = n * (t + 1) / nthreads;
        started[t] = pthread_create(&tid[t], NULL, dot_worker, &jobs[t]) == 0;
        if (!started[t])
            dot_worker(&jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) {
        if (started[t])
            pthread_join(tid[t], NULL);
        acc_merge(out, &jobs[t].acc);
    }
    free(started);
    free(tid);
    free(jobs);
}

double orc_dot_exact(int64_t n, const double *a, const double *b, int nthreads)
{
    orc_acc acc;
    exact_acc_into(&acc, n, a, b, nthreads);
    return acc_round(&acc);
}

/*
 * The exact sum as a signed big integer: out[k] (k < ORC_LIMBS) are the
 * base-2^32 limbs of |sum| * 2^2148, *neg_sign its sign.  Returns -1 when an
 * operand is non-finite, else the limb count.  Used by the tests to merge
 * partial sums from a split index range and to check rounding independently.
 */
int orc_dot_exact_fixed(int64_t n, const double *a, const double *b, uint32_t *out, int *neg_sign)
{
    orc_acc acc;
    exact_acc_into(&acc, n, a, b, 1);
    if (acc.nonfinite)
        return -1;
    acc_signed(&acc, neg_sign, out);
    return ORC_LIMBS;
}

/* round a signed big integer given as limbs (the format above) */
double orc_round_fixed(const uint32_t *limbs, int neg_sign)
{
    return round_mag(neg_sign, limbs);
}

double orc_dot_plain(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++)
        s = fma(a[i], b[i], s);
    return s;
}

/* y = A x with the fixed fma row order */
void orc_spmv(int32_t n, const int32_t *rp, const int32_t *ci, const double *v, const double *x, double *y)
{
    for (int32_t i = 0; i < n; i++) {
        double acc = 0.0;
        for (int32_t k = rp[i]; k < rp[i + 1]; k++)
            acc = fma(v[k], x[ci[k]], acc);
        y[i] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* solver                                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t n;
    const int32_t *rp, *ci;
    const double *v;
    int mode, nthreads;
    int32_t rr_period;
} orc_sys;

static double dotm(const orc_sys *S, const double *a, const double *b)
{
    if (S->mode == ORC_EXACT)
        return orc_dot_exact(S->n, a, b, S->nthreads);
    return orc_dot_plain(S->n, a, b);
}

static int fin(double a) { return is_finite_bits(a); }

/* ||b - A x||_2 / normb with the fixed SpMV and an exact dot; normb is the
   correctly rounded ||b||_2 (1 when b = 0) */
static double true_relres(const orc_sys *S, const double *b, const double *x, double normb, double *tmp)
{
    orc_spmv(S->n, S->rp, S->ci, S->v, x, tmp);
    for (int32_t i = 0; i < S->n; i++)
        tmp[i] = b[i] - tmp[i];
    double rr = orc_dot_exact(S->n, tmp, tmp, S->nthreads);
    return sqrt(rr) / normb;
}

typedef struct {
    double *hist;
    int32_t cap, len;
    double *trace;       /* per iteration: alpha_i, omega_i, beta_i, res_{i+1} */
    int32_t trace_cap;
} orc_log;

static void log_res(orc_log *L, int32_t k, double res)
{
    if (L->hist && k < L->cap)
        L->hist[k] = res;
    if (k + 1 > L->len)
        L->len = k + 1;
}

static void log_trace(orc_log *L, int32_t i, double a, double om, double be, double res)
{
    if (L->trace && i < L->trace_cap) {
        L->trace[4 * i + 0] = a;
        L->trace[4 * i + 1] = om;
        L->trace[4 * i + 2] = be;
        L->trace[4 * i + 3] = res;
    }
}

/*
 * Stop test R6.  Returns 1 when the solve is converged; may tighten *target.
 */
static int stop_test(const orc_sys *S, double res, double tol, double *target, const double *b,
                     const double *x, double *tmp, double *trueres)
{
    if (!(res <= *target))
        return 0;
    double normbt = sqrt(orc_dot_exact(S->n, b, b, S->nthreads));
    if (normbt == 0.0)
        normbt = 1.0;
    double tr = true_relres(S, b, x, normbt, tmp);
    *trueres = tr;
    if (tr <= tol)
        return 1;
    *target = tol * (tol / tr);
    return 0;
}

/* Algorithm 1 (BiCGStab) */
static int solve_bicgstab(const orc_sys *S, const double *b, double *x, double tol, int32_t maxit,
                          orc_log *L, int32_t *iters, double *relres)
{
    int32_t n = S->n;
    double *r0 = calloc((size_t)n, 8), *r = calloc((size_t)n, 8), *p = calloc((size_t)n, 8);
    double *s = calloc((size_t)n, 8), *q = calloc((size_t)n, 8), *y = calloc((size_t)n, 8);
    double *tmp = calloc((size_t)n, 8);
    int status = ORC_MAXIT;
    double trueres = NAN;
    *iters = 0;

    /* r_0 := b - A x_0 ; p_0 := r_0 */
    orc_spmv(n, S->rp, S->ci, S->v, x, tmp);
    for (int32_t i = 0; i < n; i++)
        r0[i] = b[i] - tmp[i];
    memcpy(r, r0, (size_t)n * 8);
    memcpy(p, r0, (size_t)n * 8);
    double bb = dotm(S, b, b);
    double rho = dotm(S, r0, r0);
    double normb = sqrt(bb);
    if (normb == 0.0)
        normb = 1.0;
    double res = sqrt(rho) / normb;
    double target = tol;
    log_res(L, 0, res);
    *relres = res;
    if (!fin(bb) || !fin(rho)) {
        status = ORC_NONFINITE;
        goto done;
    }
    if (stop_test(S, res, tol, &target, b, x, tmp, &trueres)) {
        status = ORC_CONVERGED;
        goto done;
    }
    for (int32_t it = 0; it < maxit; it++) {
        /* s_i := A p_i ; a_i := (r_0, r_i) / (r_0, s_i) */
        orc_spmv(n, S->rp, S->ci, S->v, p, s);
        double rs = dotm(S, r0, s);
        if (!fin(rs)) {
            status = ORC_NONFINITE;
            goto done;
        }
        double alpha = rho / rs;
        if (!fin(alpha)) {
            status = ORC_BREAKDOWN;
            goto done;
        }
        /* q_i := r_i - a_i s_i ; y_i := A q_i */
        for (int32_t i = 0; i < n; i++)
            q[i] = fma(-alpha, s[i], r[i]);
        orc_spmv(n, S->rp, S->ci, S->v, q, y);
        /* omega_i := (q_i, y_i) / (y_i, y_i) */
        double qy = dotm(S, q, y);
        double yy = dotm(S, y, y);
        if (!fin(qy) || !fin(yy)) {
            status = ORC_NONFINITE;
            goto done;
        }
        double omega = (yy == 0.0) ? 0.0 : qy / yy;
        /* x_{i+1} := x_i + a_i p_i + omega_i q_i ; r_{i+1} := q_i - omega_i y_i */
        for (int32_t i = 0; i < n; i++) {
            x[i] = fma(omega, q[i], fma(alpha, p[i], x[i]));
            r[i] = fma(-omega, y[i], q[i]);
        }
        double rho_new = dotm(S, r0, r);
        double rr = dotm(S, r, r);
        if (!fin(rho_new) || !fin(rr)) {
            status = ORC_NONFINITE;
            goto done;
        }
        *iters = it + 1;
        res = sqrt(rr) / normb;
        log_res(L, it + 1, res);
        *relres = res;
        double beta = NAN;
        if (stop_test(S, res, tol, &target, b, x, tmp, &trueres)) {
            log_trace(L, it, alpha, omega, beta, res);
            status = ORC_CONVERGED;
            goto done;
        }
        /* beta_i := (a_i / omega_i) (r_0, r_{i+1}) / (r_0, r_i) */
        if (omega != 0.0)
            beta = (alpha / omega) * (rho_new / rho);
        log_trace(L, it, alpha, omega, beta, res);
        if (omega == 0.0 || !fin(beta) || rho_new == 0.0) {
            status = ORC_BREAKDOWN;
            goto done;
        }
        /* p_{i+1} := r_{i+1} + beta_i (p_i - omega_i s_i) */
        for (int32_t i = 0; i < n; i++)
            p[i] = fma(beta, fma(-omega, s[i], p[i]), r[i]);
        rho = rho_new;
    }
    status = ORC_MAXIT;
done:
    free(r0); free(r); free(p); free(s); free(q); free(y); free(tmp);
    return status;
}

/* Algorithm 2 (p-BiCGStab) */
static int solve_pipelined(const orc_sys *S, const double *b, double *x, double tol, int32_t maxit,
                           orc_log *L, int32_t *iters, double *relres)
{
    int32_t n = S->n;
    double *r0 = calloc((size_t)n, 8), *r = calloc((size_t)n, 8), *w = calloc((size_t)n, 8);
    double *t = calloc((size_t)n, 8), *p = calloc((size_t)n, 8), *s = calloc((size_t)n, 8);
    double *z = calloc((size_t)n, 8), *v = calloc((size_t)n, 8), *q = calloc((size_t)n, 8);
    double *y = calloc((size_t)n, 8), *tmp = calloc((size_t)n, 8);
    int status = ORC_MAXIT;
    double trueres = NAN;
    *iters = 0;

    /* r_0 := b - A x_0 ; w_0 := A r_0 (R1) ; t_0 := A w_0 */
    orc_spmv(n, S->rp, S->ci, S->v, x, tmp);
    for (int32_t i = 0; i < n; i++)
        r0[i] = b[i] - tmp[i];
    memcpy(r, r0, (size_t)n * 8);
    orc_spmv(n, S->rp, S->ci, S->v, r0, w);
    orc_spmv(n, S->rp, S->ci, S->v, w, t);
    double bb = dotm(S, b, b);
    double rho = dotm(S, r0, r0);
    double rw = dotm(S, r0, w);
    double normb = sqrt(bb);
    if (normb == 0.0)
        normb = 1.0;
    double res = sqrt(rho) / normb;
    double target = tol;
    log_res(L, 0, res);
    *relres = res;
    if (!fin(bb) || !fin(rho) || !fin(rw)) {
        status = ORC_NONFINITE;
        goto done;
    }
    if (stop_test(S, res, tol, &target, b, x, tmp, &trueres)) {
        status = ORC_CONVERGED;
        goto done;
    }
    /* a_0 := (r_0, r_0) / (r_0, w_0) ; beta_{-1} := 0 */
    double alpha = rho / rw;
    if (!fin(alpha)) {
        status = ORC_BREAKDOWN;
        goto done;
    }
    double beta = 0.0, omega = 0.0;
    for (int32_t it = 0; it < maxit; it++) {
        if (it == 0) {
            /* R4: p_0 = r_0, s_0 = w_0, z_0 = t_0 */
            memcpy(p, r, (size_t)n * 8);
            memcpy(s, w, (size_t)n * 8);
            memcpy(z, t, (size_t)n * 8);
        } else if (S->rr_period > 0 && it % S->rr_period == 0) {
            /* R9: residual replacement -- true r, w, s, z (and t = A w) */
            orc_spmv(n, S->rp, S->ci, S->v, x, tmp);
            for (int32_t i = 0; i < n; i++)
                r[i] = b[i] - tmp[i];
            orc_spmv(n, S->rp, S->ci, S->v, r, w);
            for (int32_t i = 0; i < n; i++)
                p[i] = fma(beta, fma(-omega, s[i], p[i]), r[i]);
            orc_spmv(n, S->rp, S->ci, S->v, p, s);
            orc_spmv(n, S->rp, S->ci, S->v, s, z);
            orc_spmv(n, S->rp, S->ci, S->v, w, t);
        } else {
            /* p_i, s_i, z_i with beta_{i-1}, omega_{i-1} */
            for (int32_t i = 0; i < n; i++) {
                p[i] = fma(beta, fma(-omega, s[i], p[i]), r[i]);
                s[i] = fma(beta, fma(-omega, z[i], s[i]), w[i]);
                z[i] = fma(beta, fma(-omega, v[i], z[i]), t[i]);
            }
        }
        /* q_i := r_i - a_i s_i ; y_i := w_i - a_i z_i */
        for (int32_t i = 0; i < n; i++) {
            q[i] = fma(-alpha, s[i], r[i]);
            y[i] = fma(-alpha, z[i], w[i]);
        }
        /* v_i := A z_i */
        orc_spmv(n, S->rp, S->ci, S->v, z, v);
        /* omega_i := (q_i, y_i) / (y_i, y_i) */
        double qy = dotm(S, q, y);
        double yy = dotm(S, y, y);
        if (!fin(qy) || !fin(yy)) {
            status = ORC_NONFINITE;
            goto done;
        }
        omega = (yy == 0.0) ? 0.0 : qy / yy;
        /* x_{i+1}, r_{i+1}, w_{i+1} */
        for (int32_t i = 0; i < n; i++) {
            x[i] = fma(omega, q[i], fma(alpha, p[i], x[i]));
            r[i] = fma(-omega, y[i], q[i]);
            w[i] = fma(-omega, fma(-alpha, v[i], t[i]), y[i]);
        }
        /* t_{i+1} := A w_{i+1} */
        orc_spmv(n, S->rp, S->ci, S->v, w, t);
        double rho_new = dotm(S, r0, r);
        double rw_new = dotm(S, r0, w);
        double rs = dotm(S, r0, s);
        double rz = dotm(S, r0, z);
        double rr = dotm(S, r, r);
        if (!fin(rho_new) || !fin(rw_new) || !fin(rs) || !fin(rz) || !fin(rr)) {
            status = ORC_NONFINITE;
            goto done;
        }
        *iters = it + 1;
        res = sqrt(rr) / normb;
        log_res(L, it + 1, res);
        *relres = res;
        if (stop_test(S, res, tol, &target, b, x, tmp, &trueres)) {
            log_trace(L, it, alpha, omega, NAN, res);
            status = ORC_CONVERGED;
            goto done;
        }
        /* beta_i := (a_i/omega_i)(r_0, r_{i+1})/(r_0, r_i)
           a_{i+1} := (r_0, r_{i+1}) / ((r_0, w_{i+1}) + beta_i (r_0, s_i) - beta_i omega_i (r_0, z_i)) */
        double alpha_new = NAN;
        beta = NAN;
        if (omega != 0.0) {
            beta = (alpha / omega) * (rho_new / rho);
            double den = (rw_new + beta * rs) - (beta * omega) * rz;
            alpha_new = rho_new / den;
        }
        log_trace(L, it, alpha, omega, beta, res);
        if (omega == 0.0 || !fin(beta) || !fin(alpha_new) || rho_new == 0.0) {
            status = ORC_BREAKDOWN;
            goto done;
        }
        alpha = alpha_new;
        rho = rho_new;
    }
    status = ORC_MAXIT;
done:
    free(r0); free(r); free(w); free(t); free(p); free(s); free(z); free(v); free(q); free(y); free(tmp);
    return status;
}

/*
 * Solve A x = b from x (in: x_0, out: x).  Returns the solver status (>= 0)
 * or ORC_INVALID.  hist receives res_0 .. res_iters (up to hist_cap entries);
 * trace (optional) receives alpha_i, omega_i, beta_i, res_{i+1} per iteration.
 */
int orc_solve_rr(int32_t n, const int32_t *rp, const int32_t *ci, const double *v, const double *b, double *x,
                 double tol, int32_t maxit, int alg, int mode, int nthreads, int32_t rr_period, double *hist,
                 int32_t hist_cap, int32_t *hist_len, double *trace, int32_t trace_cap, int32_t *iters,
                 double *relres_rec, double *relres_true);

int orc_solve(int32_t n, const int32_t *rp, const int32_t *ci, const double *v, const double *b, double *x,
              double tol, int32_t maxit, int alg, int mode, int nthreads, double *hist, int32_t hist_cap,
              int32_t *hist_len, double *trace, int32_t trace_cap, int32_t *iters, double *relres_rec,
              double *relres_true)
{
    return orc_solve_rr(n, rp, ci, v, b, x, tol, maxit, alg, mode, nthreads, 0, hist, hist_cap, hist_len, trace,
                        trace_cap, iters, relres_rec, relres_true);
}

/* orc_solve with residual replacement every rr_period iterations (Algorithm 2 only; 0 = none) */
int orc_solve_rr(int32_t n, const int32_t *rp, const int32_t *ci, const double *v, const double *b, double *x,
                 double tol, int32_t maxit, int alg, int mode, int nthreads, int32_t rr_period, double *hist,
                 int32_t hist_cap, int32_t *hist_len, double *trace, int32_t trace_cap, int32_t *iters,
                 double *relres_rec, double *relres_true)
{
    if (rr_period < 0 || (rr_period > 0 && alg != ORC_PIPELINED))
        return ORC_INVALID;
    if (n < 1 || !rp || !ci || !v || !b || !x || !(tol > 0.0) || maxit < 0)
        return ORC_INVALID;
    if (alg != ORC_BICGSTAB && alg != ORC_PIPELINED)
        return ORC_INVALID;
    if (mode != ORC_PLAIN && mode != ORC_EXACT)
        return ORC_INVALID;
    if (rp[0] != 0)
        return ORC_INVALID;
    for (int32_t i = 0; i < n; i++)
        if (rp[i + 1] < rp[i])
            return ORC_INVALID;
    for (int32_t k = 0; k < rp[n]; k++)
        if (ci[k] < 0 || ci[k] >= n)
            return ORC_INVALID;
    orc_sys S = { n, rp, ci, v, mode, nthreads, rr_period };
    orc_log L = { hist, hist_cap, 0, trace, trace_cap };
    double rel = NAN;
    int32_t it = 0;
    int st = (alg == ORC_BICGSTAB) ? solve_bicgstab(&S, b, x, tol, maxit, &L, &it, &rel)
                                   : solve_pipelined(&S, b, x, tol, maxit, &L, &it, &rel);
    if (iters)
        *iters = it;
    if (hist_len)
        *hist_len = L.len < hist_cap ? L.len : hist_cap;
    if (relres_rec)
        *relres_rec = rel;
    if (relres_true) {
        double normbt = sqrt(orc_dot_exact(n, b, b, nthreads));
        if (normbt == 0.0)
            normbt = 1.0;
        double *tmp = calloc((size_t)n, 8);
        *relres_true = true_relres(&S, b, x, normbt, tmp);
        free(tmp);
    }
    return st;
}

/*
 * Right Jacobi preconditioning, M = diag(A) (the preconditioned variant the
 * paper mentions in Section 2; its experiments are unpreconditioned).  With
 * a diagonal M, Algorithm 1 or 2 on A M^{-1} y = b and x = M^{-1} y keeps the
 * true residual b - A x in the recurrences.  Reading: d_j is the sum, in
 * stored order, of row j's entries in column j (INVALID if zero, non-finite
 * or absent); A M^{-1} has entries v_k / d_{col_k}, one IEEE division each;
 * y0_j = x0_j * d_j; after the solve x_j = y_j / d_j.  Histories and both
 * relative residuals are those of the scaled system.
 */
int orc_solve_jacobi(int32_t n, const int32_t *rp, const int32_t *ci, const double *v, const double *b, double *x,
                     double tol, int32_t maxit, int alg, int mode, int nthreads, int32_t rr_period, double *hist,
                     int32_t hist_cap, int32_t *hist_len, double *trace, int32_t trace_cap, int32_t *iters,
                     double *relres_rec, double *relres_true)
{
    if (n < 1 || !rp || !ci || !v || !x)
        return ORC_INVALID;
    if (rp[0] != 0)
        return ORC_INVALID;
    for (int32_t i = 0; i < n; i++)
        if (rp[i + 1] < rp[i])
            return ORC_INVALID;
    for (int32_t k = 0; k < rp[n]; k++)
        if (ci[k] < 0 || ci[k] >= n)
            return ORC_INVALID;
    double *d = calloc((size_t)n, sizeof(double));
    double *vs = malloc(sizeof(double) * (size_t)(rp[n] > 0 ? rp[n] : 1));
    if (!d || !vs) {
        free(d);
        free(vs);
        return ORC_INVALID;
    }
    int bad = 0;
    for (int32_t i = 0; i < n && !bad; i++) {
        int found = 0;
        double s = 0.0;
        for (int32_t k = rp[i]; k < rp[i + 1]; k++)
            if (ci[k] == i) {
                s = found ? s + v[k] : v[k];
                found = 1;
            }
        if (!found || s == 0.0 || !fin(s))
            bad = 1;
        d[i] = s;
    }
    int st = ORC_INVALID;
    if (!bad) {
        for (int32_t k = 0; k < rp[n]; k++)
            vs[k] = v[k] / d[ci[k]];
        for (int32_t j = 0; j < n; j++)
            x[j] = x[j] * d[j];
        st = orc_solve_rr(n, rp, ci, vs, b, x, tol, maxit, alg, mode, nthreads, rr_period, hist, hist_cap, hist_len,
                          trace, trace_cap, iters, relres_rec, relres_true);
        if (st >= 0)
            for (int32_t j = 0; j < n; j++)
                x[j] = x[j] / d[j];
    }
    free(d);
    free(vs);
    return st;
}
