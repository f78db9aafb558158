/*
 * frg_oracle.c -- plain, slow, FP64 CPU oracle for the one-loop fRG flow of the
 * single-impurity Anderson model (SIAM) in Matsubara frequencies.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * path under paper_1510_07799_gb300/csrc.
 *
 * What it computes (the paper, Sec. 2 Eq. 1, states the problem as an ODE
 * dV/dg = F[V; g] for a flat array of discretised correlation functions, whose
 * right-hand side is built from three one-loop diagrams, Sec. 4; the flow of the
 * self-energy is the "straight forward" extension named in Sec. 2).  The SIAM
 * instance, the Omega-scheme cutoff and the frequency parametrisation are not
 * in the paper; the reading used here is:
 *
 *   G0^{-1}(iw) = iw - et + i Delta sgn(w),  et = eps_d + U/2  (Hartree U/2 absorbed)
 *   Theta_L(w)  = w^2 / (w^2 + L^2)          (Omega scheme)
 *   Theta_L     = 1 / sqrt(L)                (interaction flow, cutoff = 1: the bare
 *                 propagator sqrt(g) G0 with g = 1/L; L = 1 is the full model)
 *   G_L(w)      = 1 / (Theta^{-1} G0^{-1} - Sigma)
 *   S_L(w)      = dG/dL at fixed Sigma = -G^2 (d Theta^{-1}/dL) G0^{-1}
 *               (Omega: -G^2 (2L/w^2) G0^{-1}; interaction flow: -G^2 G0^{-1} / (2 sqrt L))
 *   Lb(a,b)     = S(a) G(b) + G(a) S(b)                      (bubble weight)
 *
 * V(k1,k2,k3) is the up-down vertex (k1 up-in, k2 down-in, k3 up-out,
 * k4 = k1+k2-k3 down-out).  Frequencies are indices i in [0,N) with
 * w_i = (2(i - N/2) + 1) pi T; index arithmetic is additive (i4 = i1+i2-i3).
 * Box rule: V is the stored value when all four indices lie in [0,N), else the
 * bare U.  Internal sums run over p with both internal frequencies in [0,N).
 *
 * d/dl with l = ln L (so d/dl = L d/dL):
 *   pp  (s = k1+k2):  Tpp  = -T sum_p V(k1,k2,p) Lb(p,s-p) V(p,s-p,k3)
 *   dph (t = k3-k1):  Tdph = +T sum_p Lb(p,p-t) [2 V(k1,p,k3) V(p-t,k2,p)
 *                                  - V(k1,p,p-t) V(p-t,k2,p) - V(k1,p,k3) V(p-t,k2,k4)]
 *   xph (Q = k2-k3):  Txph = -T sum_p V(k1,p+Q,p) Lb(p,p+Q) V(p,k2,k3)
 *   dV/dl      = L (Tpp + Tdph + Txph)
 *   dSigma/dl  = L T sum_p S(p) [2 V(w,p,w) - V(w,p,p)]
 *
 * Every sum above is evaluated literally, entry by entry; there is no
 * transfer-major reordering and no matrix product.
 *
 * Frequency-box tails (mask bit 4, an option beyond the paper): the internal
 * sums above run over every p of a window of TAIL_FACTOR * N Matsubara indices
 * centred on the box (both internal frequencies in the window) instead of the
 * box; vertices keep the box rule (bare U as soon as an index leaves the box)
 * and the propagators outside the box take Sigma = 0 (the flowing self-energy
 * lives on the box only).  The window is a truncation of the infinite sum:
 * the pp and xph bubble weights decay like 1/w^4 beyond it, S like 1/w^3.
 *
 * The integrator is the Dormand-Prince 5(4) pair (explicit, 7 stages, first
 * same as last), the explicit stepper family the paper uses (Sec. 2; Sec. 4
 * counts seven rhs evaluations for the first step).  Its coefficients are the
 * published Dormand-Prince table; the controller is the standard
 * max-norm one with safety 0.9, step factor clamped to [0.2, 5], exponent -1/5.
 *
 * Parity: pinned by tests against second-order perturbation theory, the exact
 * single-channel ladder solutions, a brute-force spin-resolved one-loop rhs on
 * tiny grids, the crossing/reversal symmetries, the U=0 and particle-hole
 * symmetric special cases and closed-form linear ODEs.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
    double U, T, eps_d, Delta;
    int N;
    int cutoff;  /* 0: Omega scheme; 1: interaction flow */
} oracle_model;

#define TAIL_FACTOR 16   /* window of the internal sums with mask bit 4: 16 N indices */
#define MASK_TAILS 16

/* ---------------------------------------------------------------- model --- */

static double w_of(const oracle_model *m, int i)
{
    return (2.0 * (double)(i - m->N / 2) + 1.0) * M_PI * m->T;
}

static cplx g0inv(const oracle_model *m, int i)
{
    double w = w_of(m, i);
    double et = m->eps_d + 0.5 * m->U;
    double sg = (w > 0.0) ? 1.0 : -1.0;
    return I * w - et + I * m->Delta * sg;
}

/* G_L and S_L at frequency index i (any integer), self-energy sg. */
static void propagator_at(const oracle_model *m, double L, int i, cplx sg, cplx *g_out, cplx *s_out)
{
    double w = w_of(m, i);
    double thinv = m->cutoff ? sqrt(L) : 1.0 + (L * L) / (w * w);
    double dthinv = m->cutoff ? 0.5 / sqrt(L) : 2.0 * L / (w * w);
    cplx gi = g0inv(m, i);
    cplx g = 1.0 / (thinv * gi - sg);
    *g_out = g;
    *s_out = -g * g * dthinv * gi;
}

/* G_L and S_L for every in-box frequency. sigma may be NULL (Sigma = 0). */
static void propagators(const oracle_model *m, double L, const cplx *sigma,
                        cplx *G, cplx *S)
{
    for (int i = 0; i < m->N; ++i) {
        double w = w_of(m, i);
        double thinv = m->cutoff ? sqrt(L) : 1.0 + (L * L) / (w * w);
        double dthinv = m->cutoff ? 0.5 / sqrt(L) : 2.0 * L / (w * w);
        cplx gi = g0inv(m, i);
        cplx sg = sigma ? sigma[i] : 0.0;
        cplx g = 1.0 / (thinv * gi - sg);
        G[i] = g;
        S[i] = -g * g * dthinv * gi;
    }
}

int oracle_propagators(const oracle_model *m, double L, const double *sigma,
                       double *G, double *S)
{
    propagators(m, L, (const cplx *)sigma, (cplx *)G, (cplx *)S);
    return 0;
}

/* ------------------------------------------------------------------ rhs --- */

typedef struct {
    const oracle_model *m;
    const cplx *gamma;
    const cplx *G, *S;
    /* tails: propagators on the window [lo, lo + W) of frequency indices */
    int lo, W;
    const cplx *Gw, *Sw;
} vctx;

static inline cplx Vget(const vctx *c, int i1, int i2, int i3)
{
    int N = c->m->N;
    int i4 = i1 + i2 - i3;
    if (i1 < 0 || i1 >= N || i2 < 0 || i2 >= N || i3 < 0 || i3 >= N ||
        i4 < 0 || i4 >= N)
        return c->m->U;
    return c->gamma[((size_t)i1 * N + i2) * N + i3];
}

static inline cplx Lb(const vctx *c, int a, int b)
{
    return c->S[a] * c->G[b] + c->G[a] * c->S[b];
}

static inline int inbox(int N, int i) { return i >= 0 && i < N; }

static inline int inwin(const vctx *c, int i) { return i >= c->lo && i < c->lo + c->W; }

/* bubble weight for window indices a, b */
static inline cplx Lbw(const vctx *c, int a, int b)
{
    int x = a - c->lo, y = b - c->lo;
    return c->Sw[x] * c->Gw[y] + c->Gw[x] * c->Sw[y];
}

/* The same channel sums with the internal loops over the window (tails). */
static cplx rhs_entry_tails(const vctx *c, double L, int mask, int i1, int i2, int i3)
{
    const oracle_model *m = c->m;
    int s = i1 + i2, t = i3 - i1, Q = i2 - i3, i4 = i1 + i2 - i3;
    int lo = c->lo, hi = c->lo + c->W;
    cplx pp = 0.0, dph = 0.0, xph = 0.0;
    if (mask & 1) {
        for (int p = lo; p < hi; ++p) {
            int q = s - p;
            if (!inwin(c, q)) continue;
            pp += Vget(c, i1, i2, p) * Lbw(c, p, q) * Vget(c, p, q, i3);
        }
        pp *= -m->T;
    }
    if (mask & 2) {
        for (int p = lo; p < hi; ++p) {
            int r = p - t;
            if (!inwin(c, r)) continue;
            cplx a = Vget(c, i1, p, i3);
            cplx term = 2.0 * a * Vget(c, r, i2, p)
                      - Vget(c, i1, p, r) * Vget(c, r, i2, p)
                      - a * Vget(c, r, i2, i4);
            dph += Lbw(c, p, r) * term;
        }
        dph *= m->T;
    }
    if (mask & 4) {
        for (int p = lo; p < hi; ++p) {
            int r = p + Q;
            if (!inwin(c, r)) continue;
            xph += Vget(c, i1, r, p) * Lbw(c, p, r) * Vget(c, p, i2, i3);
        }
        xph *= -m->T;
    }
    return L * (pp + dph + xph);
}

static cplx rhs_sigma_tails(const vctx *c, double L, int i)
{
    cplx acc = 0.0;
    for (int p = c->lo; p < c->lo + c->W; ++p)
        acc += c->Sw[p - c->lo] * (2.0 * Vget(c, i, p, i) - Vget(c, i, p, p));
    return L * c->m->T * acc;
}

/* Window propagators (tails): Sigma from the box, 0 outside. */
static int window_setup(vctx *c, double L, const cplx *sigma, cplx **Gw, cplx **Sw)
{
    int N = c->m->N;
    c->W = TAIL_FACTOR * N;
    c->lo = -(c->W - N) / 2;
    *Gw = malloc(sizeof(cplx) * c->W);
    *Sw = malloc(sizeof(cplx) * c->W);
    if (!*Gw || !*Sw) return -1;
    for (int x = 0; x < c->W; ++x) {
        int i = c->lo + x;
        cplx sg = (sigma && inbox(N, i)) ? sigma[i] : 0.0;
        propagator_at(c->m, L, i, sg, &(*Gw)[x], &(*Sw)[x]);
    }
    c->Gw = *Gw;
    c->Sw = *Sw;
    return 0;
}

/* d/dl of one vertex entry; mask bit0 pp, bit1 dph, bit2 xph */
static cplx rhs_entry(const vctx *c, double L, int mask, int i1, int i2, int i3)
{
    const oracle_model *m = c->m;
    int N = m->N;
    int s = i1 + i2, t = i3 - i1, Q = i2 - i3, i4 = i1 + i2 - i3;
    cplx pp = 0.0, dph = 0.0, xph = 0.0;
    if (mask & 1) {
        for (int p = 0; p < N; ++p) {
            int q = s - p;
            if (!inbox(N, q)) continue;
            pp += Vget(c, i1, i2, p) * Lb(c, p, q) * Vget(c, p, q, i3);
        }
        pp *= -m->T;
    }
    if (mask & 2) {
        for (int p = 0; p < N; ++p) {
            int r = p - t;
            if (!inbox(N, r)) continue;
            cplx a = Vget(c, i1, p, i3);
            cplx term = 2.0 * a * Vget(c, r, i2, p)
                      - Vget(c, i1, p, r) * Vget(c, r, i2, p)
                      - a * Vget(c, r, i2, i4);
            dph += Lb(c, p, r) * term;
        }
        dph *= m->T;
    }
    if (mask & 4) {
        for (int p = 0; p < N; ++p) {
            int r = p + Q;
            if (!inbox(N, r)) continue;
            xph += Vget(c, i1, r, p) * Lb(c, p, r) * Vget(c, p, i2, i3);
        }
        xph *= -m->T;
    }
    return L * (pp + dph + xph);
}

static cplx rhs_sigma(const vctx *c, double L, int i)
{
    const oracle_model *m = c->m;
    cplx acc = 0.0;
    for (int p = 0; p < m->N; ++p)
        acc += c->S[p] * (2.0 * Vget(c, i, p, i) - Vget(c, i, p, p));
    return L * m->T * acc;
}

static int g_threads = 0;

void oracle_set_threads(int n) { g_threads = n; }

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Full rhs (d/dl) for rows i1 in [k1_begin, k1_end): writes dgamma for those
 * rows (other rows untouched) and, if dsigma != NULL and mask bit3 is set,
 * the whole dSigma (else dSigma = 0).  gamma, sigma, dgamma, dsigma are
 * complex128 arrays, interleaved re/im, gamma index ((i1*N)+i2)*N+i3.
 */
int oracle_rhs_rows(const oracle_model *m, double L, const double *gamma,
                    const double *sigma, int mask, int k1_begin, int k1_end,
                    double *dgamma, double *dsigma)
{
    int N = m->N;
    cplx *G = malloc(sizeof(cplx) * N), *S = malloc(sizeof(cplx) * N);
    if (!G || !S) { free(G); free(S); return -1; }
    propagators(m, L, (const cplx *)sigma, G, S);
    vctx c = {m, (const cplx *)gamma, G, S, 0, 0, NULL, NULL};
    cplx *Gw = NULL, *Sw = NULL;
    const int tails = (mask & MASK_TAILS) != 0;
    if (tails && window_setup(&c, L, (const cplx *)sigma, &Gw, &Sw)) {
        free(G); free(S); free(Gw); free(Sw);
        return -1;
    }
    cplx *dg = (cplx *)dgamma;
#ifdef _OPENMP
    int nt = oracle_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int i1 = k1_begin; i1 < k1_end; ++i1)
        for (int i2 = 0; i2 < N; ++i2)
            for (int i3 = 0; i3 < N; ++i3)
                dg[((size_t)i1 * N + i2) * N + i3] =
                    tails ? rhs_entry_tails(&c, L, mask, i1, i2, i3) : rhs_entry(&c, L, mask, i1, i2, i3);
    if (dsigma) {
        cplx *ds = (cplx *)dsigma;
        for (int i = 0; i < N; ++i)
            ds[i] = (mask & 8) ? (tails ? rhs_sigma_tails(&c, L, i) : rhs_sigma(&c, L, i)) : 0.0;
    }
    free(G); free(S); free(Gw); free(Sw);
    return 0;
}

int oracle_rhs(const oracle_model *m, double L, const double *gamma,
               const double *sigma, int mask, double *dgamma, double *dsigma)
{
    return oracle_rhs_rows(m, L, gamma, sigma, mask, 0, m->N, dgamma, dsigma);
}

/* rhs at an explicit list of entries idx[3*j + {0,1,2}] = (i1,i2,i3). */
int oracle_rhs_entries(const oracle_model *m, double L, const double *gamma,
                       const double *sigma, int mask, int count, const int *idx,
                       double *out)
{
    int N = m->N;
    cplx *G = malloc(sizeof(cplx) * N), *S = malloc(sizeof(cplx) * N);
    if (!G || !S) { free(G); free(S); return -1; }
    propagators(m, L, (const cplx *)sigma, G, S);
    vctx c = {m, (const cplx *)gamma, G, S, 0, 0, NULL, NULL};
    cplx *Gw = NULL, *Sw = NULL;
    const int tails = (mask & MASK_TAILS) != 0;
    if (tails && window_setup(&c, L, (const cplx *)sigma, &Gw, &Sw)) {
        free(G); free(S); free(Gw); free(Sw);
        return -1;
    }
    cplx *o = (cplx *)out;
#ifdef _OPENMP
    int nt = oracle_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
#endif
    for (int j = 0; j < count; ++j)
        o[j] = tails ? rhs_entry_tails(&c, L, mask, idx[3 * j], idx[3 * j + 1], idx[3 * j + 2])
                     : rhs_entry(&c, L, mask, idx[3 * j], idx[3 * j + 1], idx[3 * j + 2]);
    free(G); free(S); free(Gw); free(Sw);
    return 0;
}

/* ------------------------------------------------------------ DP5 (4) --- */

/* Dormand-Prince 5(4) coefficients (published table). */
static const double DP_C[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
/* 5th-order weights are the last row of A (first same as last); 4th-order: */
static const double DP_BSTAR[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640,
                                   -92097.0 / 339200, 187.0 / 2100, 1.0 / 40};

void oracle_dp5_tableau(double *c, double *a, double *b, double *bstar)
{
    for (int i = 0; i < 7; ++i) {
        c[i] = DP_C[i];
        for (int j = 0; j < 6; ++j) a[i * 6 + j] = DP_A[i][j];
        b[i] = (i < 6) ? DP_A[6][i] : 0.0;
        bstar[i] = DP_BSTAR[i];
    }
}

typedef int (*oracle_rhs_fn)(double t, const double *y, double *dydt, void *ctx);

typedef struct {
    double t;        /* final t reached */
    double h;        /* next step size proposal */
    long accepted, rejected, rhs_evals;
    int status;      /* 0 ok, -5 not converged, -4 non-finite */
    long first_step_evals; /* evaluations spent until the first accepted step */
} oracle_dp5_stats;

/*
 * Integrate y' = f(t, y) from t0 to t1 (either direction) with DP5(4).
 * err = max_i |e_i| / (atol + rtol max(|y_i|, |ynew_i|)); accept if err <= 1.
 * step factor = clamp(0.9 err^{-1/5}, 0.2, 5); the last step is clipped to t1.
 * If fixed_h != 0 the controller is bypassed and steps of fixed_h are taken
 * (last one clipped), used by the order tests.
 */
int oracle_dp5(long n, double *y, double t0, double t1, double h0, double rtol,
               double atol, long max_steps, double fixed_h, oracle_rhs_fn f,
               void *ctx, oracle_dp5_stats *st)
{
    double *k[7], *ys = malloc(sizeof(double) * n), *yn = malloc(sizeof(double) * n);
    int ok = ys && yn;
    for (int i = 0; i < 7; ++i) { k[i] = malloc(sizeof(double) * n); ok = ok && k[i]; }
    memset(st, 0, sizeof(*st));
    if (!ok) {
        for (int i = 0; i < 7; ++i) free(k[i]);
        free(ys); free(yn);
        return -2;
    }
    double dir = (t1 >= t0) ? 1.0 : -1.0;
    double t = t0;
    double h = fixed_h != 0.0 ? fixed_h : h0;
    if (h * dir <= 0) h = -h;
    int have_k1 = 0, status = 0;
    long steps = 0;
    while ((t1 - t) * dir > 0) {
        if (steps++ >= max_steps) { status = -5; break; }
        int last = 0;
        if ((t + h - t1) * dir >= 0) { h = t1 - t; last = 1; }
        if (!have_k1) {
            if (f(t, y, k[0], ctx)) { status = -3; break; }
            st->rhs_evals++;
            have_k1 = 1;
        }
        for (int s = 1; s < 7; ++s) {
            for (long i = 0; i < n; ++i) {
                double acc = 0.0;
                for (int j = 0; j < s; ++j) acc += DP_A[s][j] * k[j][i];
                ys[i] = y[i] + h * acc;
            }
            if (f(t + DP_C[s] * h, ys, k[s], ctx)) { status = -3; break; }
            st->rhs_evals++;
        }
        if (status) break;
        /* ys now holds the 5th-order solution (stage 7 input = b weights) */
        memcpy(yn, ys, sizeof(double) * n);
        double err = 0.0;
        int finite = 1;
        for (long i = 0; i < n; ++i) {
            double e = 0.0;
            for (int j = 0; j < 7; ++j) {
                double bj = (j < 6) ? DP_A[6][j] : 0.0;
                e += (bj - DP_BSTAR[j]) * k[j][i];
            }
            e *= h;
            double sc = atol + rtol * fmax(fabs(y[i]), fabs(yn[i]));
            double r = fabs(e) / sc;
            if (!isfinite(r) || !isfinite(yn[i])) finite = 0;
            if (r > err) err = r;
        }
        if (!finite) { status = -4; break; }
        if (fixed_h != 0.0 || err <= 1.0) {
            t = last ? t1 : t + h;
            memcpy(y, yn, sizeof(double) * n);
            double *tmp = k[0]; k[0] = k[6]; k[6] = tmp; /* first same as last */
            st->accepted++;
            if (st->accepted == 1) st->first_step_evals = st->rhs_evals;
            if (fixed_h == 0.0) {
                double fac = (err == 0.0) ? 5.0 : 0.9 * pow(err, -0.2);
                if (fac > 5.0) fac = 5.0;
                if (fac < 0.2) fac = 0.2;
                h *= fac;
            } else {
                h = fixed_h;
            }
        } else {
            double fac = 0.9 * pow(err, -0.2);
            if (fac < 0.2) fac = 0.2;
            h *= fac;
            st->rejected++;
            if (fabs(h) < 1e-14 * fmax(1.0, fabs(t))) { status = -5; break; }
        }
    }
    st->t = t;
    st->h = h;
    st->status = status;
    for (int i = 0; i < 7; ++i) free(k[i]);
    free(ys); free(yn);
    return status;
}

/* ------------------------------------------------------------- the flow --- */

typedef struct {
    const oracle_model *m;
    int mask;
} flow_ctx;

static int flow_rhs(double l, const double *y, double *dydt, void *vctx_)
{
    const flow_ctx *fc = (const flow_ctx *)vctx_;
    const oracle_model *m = fc->m;
    size_t N3 = (size_t)m->N * m->N * m->N;
    double L = exp(l);
    return oracle_rhs(m, L, y, y + 2 * N3, fc->mask, dydt, dydt + 2 * N3);
}

/*
 * Flow gamma (N^3 complex) and sigma (N complex) from Lambda0 to Lambda_f in
 * l = ln Lambda with DP5, in place.  h0 is the initial step in l (negative).
 */
int oracle_flow(const oracle_model *m, int mask, double Lambda0, double Lambda_f,
                double rtol, double atol, double h0, long max_steps,
                double *gamma, double *sigma, oracle_dp5_stats *st)
{
    size_t N3 = (size_t)m->N * m->N * m->N;
    long n = (long)(2 * N3 + 2 * (size_t)m->N);
    double *y = malloc(sizeof(double) * n);
    if (!y) return -2;
    memcpy(y, gamma, sizeof(double) * 2 * N3);
    memcpy(y + 2 * N3, sigma, sizeof(double) * 2 * m->N);
    flow_ctx fc = {m, mask};
    int rc = oracle_dp5(n, y, log(Lambda0), log(Lambda_f), h0, rtol, atol,
                        max_steps, 0.0, flow_rhs, &fc, st);
    memcpy(gamma, y, sizeof(double) * 2 * N3);
    memcpy(sigma, y + 2 * N3, sizeof(double) * 2 * m->N);
    free(y);
    return rc;
}

/* Observables at scale L: Sigma(pi T), Z, U_eff = V(0,0,0) in n-notation, and
 * the in-box occupation per spin (informational only). out[0..5] =
 * {Re Sigma(piT), Im Sigma(piT), Z, Re Ueff, Im Ueff, n}. */
int oracle_observables(const oracle_model *m, double L, const double *gamma,
                       const double *sigma, double *out)
{
    int N = m->N, h = N / 2;
    const cplx *sg = (const cplx *)sigma;
    const cplx *gm = (const cplx *)gamma;
    cplx s0 = sg[h];
    double w0 = M_PI * m->T;
    cplx ueff = gm[((size_t)h * N + h) * N + h];
    cplx *G = malloc(sizeof(cplx) * N), *S = malloc(sizeof(cplx) * N);
    if (!G || !S) { free(G); free(S); return -1; }
    propagators(m, L, sg, G, S);
    double n = 0.5;
    for (int i = 0; i < N; ++i) n += m->T * creal(G[i]);
    free(G); free(S);
    out[0] = creal(s0);
    out[1] = cimag(s0);
    out[2] = 1.0 / (1.0 - cimag(s0) / w0);
    out[3] = creal(ueff);
    out[4] = cimag(ueff);
    out[5] = n;
    return 0;
}
