/* Plain C restatement of the oracle's Wilson-clover matrix K and of textbook
 * BiCGStab, for lattices where the numpy stencil is too slow.  Test
 * infrastructure only (see oracle/__init__.py); shares nothing with the CUDA
 * library.
 *
 * K psi(x) = A(x) psi(x)
 *            - 1/2 sum_mu w_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu) s_f
 *                               + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) s_b ]
 * with A(x) the 12x12 mass+clover matrix supplied by the caller (built by the
 * numpy oracle), w = (1/xi, 1/xi, 1/xi, 1), and s_f = -1 (s_b = -1) for hops
 * that cross the time boundary (antiperiodic fermions), else +1.
 *
 * Layouts (complex double, x fastest): links [V][4][3][3], clover [V][12][12],
 * spinors [V][4][3].  The chiral-basis gamma matrices are written out below.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const cplx GAM[4][4][4] = {
    /* gamma_1 = [[0, -i s1], [i s1, 0]] */
    {{0, 0, 0, -I}, {0, 0, -I, 0}, {0, I, 0, 0}, {I, 0, 0, 0}},
    /* gamma_2 = [[0, -i s2], [i s2, 0]] */
    {{0, 0, 0, -1}, {0, 0, 1, 0}, {0, 1, 0, 0}, {-1, 0, 0, 0}},
    /* gamma_3 = [[0, -i s3], [i s3, 0]] */
    {{0, 0, -I, 0}, {0, 0, 0, I}, {I, 0, 0, 0}, {0, -I, 0, 0}},
    /* gamma_4 = [[0, 1], [1, 0]] */
    {{0, 0, 1, 0}, {0, 0, 0, 1}, {1, 0, 0, 0}, {0, 1, 0, 0}},
};

typedef struct {
    const cplx *U;
    const cplx *A;
    int ns, nt;
    double w[4];
    int nthreads; /* threads splitting the site loop of one application (0 or 1: none) */
} op_t;

static void neighbours(const op_t *op, long s, int mu, long *fw, long *bw, double *sf, double *sb) {
    int ns = op->ns, nt = op->nt;
    int x = (int)(s % ns), y = (int)((s / ns) % ns), z = (int)((s / ((long)ns * ns)) % ns);
    int t = (int)(s / ((long)ns * ns * ns));
    int c[4] = {x, y, z, t};
    int d[4] = {ns, ns, ns, nt};
    int cf[4], cb[4];
    memcpy(cf, c, sizeof c);
    memcpy(cb, c, sizeof c);
    cf[mu] = (c[mu] + 1) % d[mu];
    cb[mu] = (c[mu] - 1 + d[mu]) % d[mu];
    *fw = (((long)cf[3] * ns + cf[2]) * ns + cf[1]) * ns + cf[0];
    *bw = (((long)cb[3] * ns + cb[2]) * ns + cb[1]) * ns + cb[0];
    *sf = (mu == 3 && t == nt - 1) ? -1.0 : 1.0;
    *sb = (mu == 3 && t == 0) ? -1.0 : 1.0;
}

/* out = K in on the sites [s0, s1). */
static void apply_K_range(const op_t *op, const cplx *in, cplx *out, long s0, long s1) {
    for (long s = s0; s < s1; ++s) {
        cplx acc[12];
        const cplx *a = op->A + s * 144;
        for (int i = 0; i < 12; ++i) {
            cplx v = 0;
            for (int j = 0; j < 12; ++j) v += a[i * 12 + j] * in[s * 12 + j];
            acc[i] = v;
        }
        for (int mu = 0; mu < 4; ++mu) {
            long fw, bw;
            double sf, sb;
            neighbours(op, s, mu, &fw, &bw, &sf, &sb);
            const cplx *uf = op->U + (s * 4 + mu) * 9;
            const cplx *ub = op->U + (bw * 4 + mu) * 9;
            cplx hf[4][3], hb[4][3];
            /* colour: U(x) psi(x+mu) and U(x-mu)^dag psi(x-mu) */
            for (int sp = 0; sp < 4; ++sp)
                for (int a2 = 0; a2 < 3; ++a2) {
                    cplx vf = 0, vb = 0;
                    for (int b = 0; b < 3; ++b) {
                        vf += uf[a2 * 3 + b] * in[fw * 12 + sp * 3 + b];
                        vb += conj(ub[b * 3 + a2]) * in[bw * 12 + sp * 3 + b];
                    }
                    hf[sp][a2] = vf * sf;
                    hb[sp][a2] = vb * sb;
                }
            /* spin: (1 - gamma) hf + (1 + gamma) hb */
            for (int sp = 0; sp < 4; ++sp)
                for (int a2 = 0; a2 < 3; ++a2) {
                    cplx v = hf[sp][a2] + hb[sp][a2];
                    for (int r = 0; r < 4; ++r) v += GAM[mu][sp][r] * (hb[r][a2] - hf[r][a2]);
                    acc[sp * 3 + a2] -= 0.5 * op->w[mu] * v;
                }
        }
        for (int i = 0; i < 12; ++i) out[s * 12 + i] = acc[i];
    }
}

typedef struct {
    const op_t *op;
    const cplx *in;
    cplx *out;
    long s0, s1;
} range_t;

static void *range_worker(void *arg) {
    const range_t *r = (const range_t *)arg;
    apply_K_range(r->op, r->in, r->out, r->s0, r->s1);
    return NULL;
}

/* out = K in; the sites are split over op->nthreads threads when asked (every site's
   arithmetic is the same either way). */
static void apply_K(const op_t *op, const cplx *in, cplx *out) {
    long V = (long)op->ns * op->ns * op->ns * op->nt;
    int nth = op->nthreads;
    if (nth <= 1) {
        apply_K_range(op, in, out, 0, V);
        return;
    }
    if (nth > 64) nth = 64;
    pthread_t th[64];
    range_t rg[64];
    for (int i = 0; i < nth; ++i) {
        rg[i].op = op;
        rg[i].in = in;
        rg[i].out = out;
        rg[i].s0 = V * i / nth;
        rg[i].s1 = V * (i + 1) / nth;
        pthread_create(&th[i], NULL, range_worker, &rg[i]);
    }
    for (int i = 0; i < nth; ++i) pthread_join(th[i], NULL);
}

static cplx dotc(const cplx *a, const cplx *b, long n) {
    cplx s = 0;
    for (long i = 0; i < n; ++i) s += conj(a[i]) * b[i];
    return s;
}

static double nrm2(const cplx *a, long n) { return sqrt(creal(dotc(a, a, n))); }

/* Textbook BiCGStab (van der Vorst 1992) from x = 0.  Returns iterations. */
static int bicgstab(const op_t *op, const cplx *b, cplx *x, double tol, int maxiter, double *relres) {
    long n = (long)op->ns * op->ns * op->ns * op->nt * 12;
    cplx *r = malloc(n * sizeof(cplx)), *rh = malloc(n * sizeof(cplx)), *p = calloc(n, sizeof(cplx));
    cplx *v = calloc(n, sizeof(cplx)), *s = malloc(n * sizeof(cplx)), *t = malloc(n * sizeof(cplx));
    memset(x, 0, n * sizeof(cplx));
    memcpy(r, b, n * sizeof(cplx));
    memcpy(rh, b, n * sizeof(cplx));
    double bn = nrm2(b, n);
    cplx rho_old = 1, alpha = 1, omega = 1;
    int it = 0;
    while (bn > 0 && it < maxiter) {
        ++it;
        cplx rho = dotc(rh, r, n);
        cplx beta = (rho / rho_old) * (alpha / omega);
        for (long i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
        apply_K(op, p, v);
        alpha = rho / dotc(rh, v, n);
        for (long i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
        if (nrm2(s, n) <= tol * bn) {
            for (long i = 0; i < n; ++i) x[i] += alpha * p[i];
            break;
        }
        apply_K(op, s, t);
        omega = dotc(t, s, n) / dotc(t, t, n);
        for (long i = 0; i < n; ++i) {
            x[i] += alpha * p[i] + omega * s[i];
            r[i] = s[i] - omega * t[i];
        }
        rho_old = rho;
        if (nrm2(r, n) <= tol * bn) break;
    }
    apply_K(op, x, t);
    for (long i = 0; i < n; ++i) t[i] = b[i] - t[i];
    *relres = bn > 0 ? nrm2(t, n) / bn : 0.0;
    free(r); free(rh); free(p); free(v); free(s); free(t);
    return it;
}

void oracle_K_apply(const double *U, const double *A, int ns, int nt, double xi,
                    const double *in, double *out) {
    op_t op = {(const cplx *)U, (const cplx *)A, ns, nt, {1.0 / xi, 1.0 / xi, 1.0 / xi, 1.0}, 1};
    apply_K(&op, (const cplx *)in, (cplx *)out);
}

typedef struct {
    const op_t *op;
    const cplx *b;
    cplx *x;
    int nrhs, maxiter, stride;
    double tol;
    int *iters;
    double *relres;
    int first;
} job_t;

static void *worker(void *arg) {
    job_t *j = (job_t *)arg;
    long n = (long)j->op->ns * j->op->ns * j->op->ns * j->op->nt * 12;
    for (int k = j->first; k < j->nrhs; k += j->stride)
        j->iters[k] = bicgstab(j->op, j->b + k * n, j->x + k * n, j->tol, j->maxiter, &j->relres[k]);
    return NULL;
}

/* nrhs independent single-threaded solves spread over nthreads threads. */
void oracle_bicgstab_batch(const double *U, const double *A, int ns, int nt, double xi,
                           const double *b, double *x, int nrhs, double tol, int maxiter,
                           int nthreads, int *iters, double *relres) {
    op_t op = {(const cplx *)U, (const cplx *)A, ns, nt, {1.0 / xi, 1.0 / xi, 1.0 / xi, 1.0}, 1};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nrhs) nthreads = nrhs;
    pthread_t th[256];
    job_t jobs[256];
    if (nthreads > 256) nthreads = 256;
    for (int i = 0; i < nthreads; ++i) {
        jobs[i] = (job_t){&op, (const cplx *)b, (cplx *)x, nrhs, maxiter, nthreads, tol, iters, relres, i};
        pthread_create(&th[i], NULL, worker, &jobs[i]);
    }
    for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
}

/* One BiCGStab solve of K x = b with the site loop of each application of K split over
   nthreads threads; returns the iteration count. */
int oracle_bicgstab_threaded(const double *U, const double *A, int ns, int nt, double xi, const double *b,
                             double *x, double tol, int maxiter, int nthreads, double *relres) {
    op_t op = {(const cplx *)U, (const cplx *)A, ns, nt, {1.0 / xi, 1.0 / xi, 1.0 / xi, 1.0}, nthreads};
    return bicgstab(&op, (const cplx *)b, (cplx *)x, tol, maxiter, relres);
}
