/*
 * rswr_oracle.c -- CPU oracle for the RSWR wave-equation hot path.
 *
 * TEST INFRASTRUCTURE.  This file is the plain, slow, obviously correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * library never does.  It shares no code, header or constant with the CUDA
 * path: every coefficient is derived here from (xa, xb, a, nx, dt).
 *
 * Build with -ffp-contract=off so that the compiler never fuses a multiply and
 * an add that the source writes separately; every fused multiply-add below is
 * an explicit call of the correctly rounded C99 fma()/fmaf().
 *
 * Contents
 *   oracle_coeffs            grid and stencil coefficients
 *   oracle_leapfrog_{f64,f32}   monolithic leapfrog ("true solution", Sec. 2.1)
 *   oracle_rswr_mask_{f64,f32}  serial RSWR, select as an index mask (Sec. 2.2-2.6, Sec. 3)
 *   oracle_rswr_paper        serial RSWR with the paper's adaptive select and
 *                            flux-exchange update (Sec. 2.3-2.6, Sec. 3)
 *   oracle_adjoint           discrete adjoint of the canonical leapfrog for a
 *                            receiver-trace cotangent (not in the paper; the
 *                            gradient workload of the project)
 *
 * Parity status of every function: pinned by tests/test_oracle_*.py (closed
 * forms, exact rational brute force, conservation, dot-product and finite
 * difference checks).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Grid spacing and stencil coefficients of the leapfrog for u_tt = a^2 u_xx
 * (paper Eq. (2.1)).  dx = (xb - xa)/(nx - 1); Courant number c = a dt / dx;
 * c2 = c*c; k = 2 - 2 c2; inv2dx = 1/(2 dx) scales a central difference into
 * the flux du/dx (paper Sec. 2.2, boundary flux waveforms).  The float
 * coefficients are the double ones rounded once, k recomputed in float. */
void oracle_coeffs(double xa, double xb, double a, int64_t nx, double dt,
                   double* c, double* c2, double* k, double* inv2dx,
                   float* c2f, float* kf, float* inv2dxf)
{
    double dx = (xb - xa) / (double)(nx - 1);
    double cc = a * dt / dx;
    *c = cc;
    *c2 = cc * cc;
    *k = 2.0 - 2.0 * (*c2);
    *inv2dx = 1.0 / (2.0 * dx);
    *c2f = (float)(*c2);
    *kf = 2.0f - 2.0f * (*c2f);
    *inv2dxf = (float)(*inv2dx);
}

/* Threads of the monolithic leapfrog's interior loop (1 = serial, the
 * default).  The updates of one level read only the previous levels, so the
 * result is the same bit for bit for any count; threads only shorten the
 * CPU timing baseline.  Effective when the file is built with -fopenmp. */
static int oracle_nthreads = 1;

void oracle_set_threads(int n) { oracle_nthreads = n < 1 ? 1 : n; }

#define REAL double
#define FMA fma
#define NAME(x) x##_f64
#include "leapfrog_body.h"
#undef REAL
#undef FMA
#undef NAME

#define REAL float
#define FMA fmaf
#define NAME(x) x##_f32
#include "leapfrog_body.h"
#undef REAL
#undef FMA
#undef NAME

/* ------------------------------------------------------------------------- */
/* Paper-literal serial RSWR (FP64).                                          */
/* ------------------------------------------------------------------------- */

static int64_t win_left(int64_t i, int64_t nx, int64_t N, int64_t el)
{
    int64_t b0 = i * nx / N;
    return b0 - el < 0 ? 0 : b0 - el;
}

static int64_t win_right(int64_t i, int64_t nx, int64_t N, int64_t er)
{
    int64_t b1 = (i + 1) * nx / N;
    return b1 - 1 + er > nx - 1 ? nx - 1 : b1 - 1 + er;
}

/*
 * One window solve over `steps` steps starting from the true state (u, w) at
 * level n0.  At an input boundary the ghost value comes from a prescribed
 * boundary flux g (Neumann transmission condition, Sec. 2.2):
 *   left end L:   u_{L-1} = u_{L+1} - 2 dx g_L
 *   right end R:  u_{R+1} = u_{R-1} + 2 dx g_R
 * gL / gR hold one flux per step (NULL means the zero-flux prediction guess of
 * Sec. 2.3).  The full trajectory of u is stored: traj[s*nx + j], s = 0..steps.
 */
static void window_solve(int form, int64_t nx, double c2, double k, double dx,
                         const double* fA, const double* fB, const double* u, const double* w,
                         int64_t L, int64_t R, int64_t n0, int64_t steps,
                         const double* gL, const double* gR,
                         double* traj, double* end_u, double* end_w, double* tmp_u, double* tmp_w)
{
    double* pu = end_u;
    double* pw = end_w;
    for (int64_t j = L; j <= R; ++j) { pu[j] = u[j]; pw[j] = w[j]; traj[j] = u[j]; }
    for (int64_t s = 0; s < steps; ++s) {
        int64_t n = n0 + s;
        for (int64_t j = L; j <= R; ++j) {
            if (j == 0) {
                tmp_u[j] = fA[n + 1];
                tmp_w[j] = dirichlet_w_f64(form, fA[n], fA[n + 1]);
            } else if (j == nx - 1) {
                tmp_u[j] = fB[n + 1];
                tmp_w[j] = dirichlet_w_f64(form, fB[n], fB[n + 1]);
            } else {
                double uL, uR;
                if (j == L) uL = gL ? pu[j + 1] - 2.0 * dx * gL[s] : pu[j + 1];
                else uL = pu[j - 1];
                if (j == R) uR = gR ? pu[j - 1] + 2.0 * dx * gR[s] : pu[j - 1];
                else uR = pu[j + 1];
                point_update_f64(form, c2, k, uL, pu[j], uR, pw[j], &tmp_u[j], &tmp_w[j]);
            }
        }
        for (int64_t j = L; j <= R; ++j) { pu[j] = tmp_u[j]; pw[j] = tmp_w[j]; traj[(s + 1) * nx + j] = pu[j]; }
    }
}

/*
 * Serial RSWR as the paper states it (Sec. 2.3-2.6; N > 2 per Sec. 3):
 *   predict: every window is advanced tau steps (tau = predictive span) from
 *       the true state with a zero input flux guess;
 *   select: on each overlap O_{i,i+1} the point span Delta T(x) is the number
 *       of steps over which the two predictions agree exactly at x; the
 *       pair's maximum span is the largest Delta T(x); the global span is the
 *       minimum over pairs (Sec. 3), capped by the Waveform Time Span Theorem
 *       (Delta T_max < Delta X_overlap / (2a), i.e. steps < (ov - 1)/(2c)) and
 *       by tau;
 *   update: every window is solved again over the selected span with its
 *       input flux set to the neighbour's predicted output flux (Sec. 2.5);
 *   combine: u = p_i on Omega_i minus the windows left of it (Sec. 2.5);
 *   redo: the next predictive span is ceil((1 + beta) Delta T_max) (Sec. 2.6),
 *       with beta taken in thousandths so that the product is exact.
 * spans[m] receives the m-th selected span; *nspans their number.
 * Returns 0 on success.
 */
int oracle_rswr_paper(int form, int64_t nx, int64_t T, double c, double c2, double k, double dx,
                      const double* fA, const double* fB, int64_t N, int64_t ov,
                      int64_t tau0, double beta, double* out0, double* out1,
                      int64_t* spans, int64_t* nspans)
{
    if (nx < 3 || T < 0 || N < 1 || ov < 2) return 1;
    int64_t el = (ov + 1) / 2, er = ov / 2;
    double cap_real = (double)(ov - 1) / (2.0 * c);
    int64_t cap = (int64_t)ceil(cap_real) - 1;
    if (cap < 1) cap = 1;
    int64_t tau = tau0 > 0 ? tau0 : ov;
    /* beta in thousandths: the next predictive span ceil((1 + beta) span) is
     * then exact integer arithmetic (in doubles, 1.1 * 50 rounds above 55) */
    int64_t beta_m = (int64_t)llround(beta * 1000.0);
    int64_t tau_max = tau > cap ? tau : cap;
    tau_max = (tau_max * (1000 + beta_m) + 999) / 1000 + 1;

    double* u = (double*)calloc(nx, sizeof(double));
    double* w = (double*)calloc(nx, sizeof(double));
    double* nu = (double*)calloc(nx, sizeof(double));
    double* nw = (double*)calloc(nx, sizeof(double));
    double* eu = (double*)calloc(nx, sizeof(double));
    double* ew = (double*)calloc(nx, sizeof(double));
    double* tu = (double*)calloc(nx, sizeof(double));
    double* tw = (double*)calloc(nx, sizeof(double));
    double* traj = (double*)calloc((size_t)N * (tau_max + 1) * nx, sizeof(double));
    double* gbuf = (double*)calloc(2 * (size_t)(tau_max + 1), sizeof(double));
    double* scratch = (double*)calloc((size_t)(tau_max + 1) * nx, sizeof(double));
    if (!u || !w || !nu || !nw || !eu || !ew || !tu || !tw || !traj || !gbuf || !scratch) {
        free(u); free(w); free(nu); free(nw); free(eu); free(ew); free(tu); free(tw);
        free(traj); free(gbuf); free(scratch);
        return 2;
    }
    init_state_f64(form, nx, fA, fB, NULL, NULL, u, w);
    int64_t m = 0;
    for (int64_t n0 = 0; n0 < T;) {
        int64_t steps = tau < T - n0 ? tau : T - n0;
        /* predict */
        for (int64_t i = 0; i < N; ++i) {
            window_solve(form, nx, c2, k, dx, fA, fB, u, w, win_left(i, nx, N, el), win_right(i, nx, N, er),
                         n0, steps, NULL, NULL, traj + (size_t)i * (tau_max + 1) * nx, eu, ew, tu, tw);
        }
        /* select */
        int64_t span = steps;
        for (int64_t i = 0; i + 1 < N; ++i) {
            const double* p1 = traj + (size_t)i * (tau_max + 1) * nx;
            const double* p2 = traj + (size_t)(i + 1) * (tau_max + 1) * nx;
            int64_t best = 0;
            for (int64_t x = win_left(i + 1, nx, N, el); x <= win_right(i, nx, N, er); ++x) {
                int64_t agree = 0;
                while (agree < steps && p1[(agree + 1) * nx + x] == p2[(agree + 1) * nx + x]) ++agree;
                if (agree > best) best = agree;
            }
            if (best < span) span = best;
        }
        if (span > cap) span = cap;
        if (span < 1) span = 1;
        /* update: solve again with the neighbours' predicted output fluxes */
        for (int64_t i = 0; i < N; ++i) {
            int64_t L = win_left(i, nx, N, el), R = win_right(i, nx, N, er);
            double* gL = NULL;
            double* gR = NULL;
            if (i > 0 && L > 0) {
                const double* pn = traj + (size_t)(i - 1) * (tau_max + 1) * nx;
                gL = gbuf;
                for (int64_t s = 0; s < span; ++s)
                    gL[s] = (pn[s * nx + L + 1] - pn[s * nx + L - 1]) / (2.0 * dx);
            }
            if (i + 1 < N && R < nx - 1) {
                const double* pn = traj + (size_t)(i + 1) * (tau_max + 1) * nx;
                gR = gbuf + (tau_max + 1);
                for (int64_t s = 0; s < span; ++s)
                    gR[s] = (pn[s * nx + R + 1] - pn[s * nx + R - 1]) / (2.0 * dx);
            }
            window_solve(form, nx, c2, k, dx, fA, fB, u, w, L, R, n0, span, gL, gR, scratch, eu, ew, tu, tw);
            /* combine: points of Omega_i not covered by a window further left */
            int64_t from = (i == 0) ? L : win_right(i - 1, nx, N, er) + 1;
            for (int64_t j = from; j <= R; ++j) { nu[j] = eu[j]; nw[j] = ew[j]; }
        }
        double* t;
        t = u; u = nu; nu = t;
        t = w; w = nw; nw = t;
        if (spans) spans[m] = span;
        ++m;
        n0 += span;
        tau = (span * (1000 + beta_m) + 999) / 1000;
        if (tau > tau_max) tau = tau_max;
    }
    if (nspans) *nspans = m;
    memcpy(out0, u, sizeof(double) * nx);
    memcpy(out1, w, sizeof(double) * nx);
    /* u / nu and w / nw were swapped a whole number of times: free the four
     * buffers through a list of their current names */
    double* bufs[4] = {u, w, nu, nw};
    for (int b = 0; b < 4; ++b) free(bufs[b]);
    free(eu); free(ew); free(tu); free(tw);
    free(traj); free(gbuf); free(scratch);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Discrete adjoint of the canonical leapfrog (FP64).                         */
/* ------------------------------------------------------------------------- */

/*
 * Forward: zero initial data, Dirichlet samples fA, fB, canonical form
 *   u^{n+1}_j = c2 (u^n_{j-1} + u^n_{j+1}) + k u^n_j - u^{n-1}_j,  u^{-1} = u^0.
 * Receiver trace y^n = u^n_{jr}, n = 0..T.  Given a cotangent wbar = dL/dy,
 * the adjoint variables lambda^n_j = dL/du^n_j (interior j) satisfy, backward
 * in time with lambda^{T+1} = lambda^{T+2} = 0 and lambda = 0 on the boundary
 * nodes,
 *   lambda^n_j = c2 (lambda^{n+1}_{j-1} + lambda^{n+1}_{j+1}) + k lambda^{n+1}_j
 *                - lambda^{n+2}_j + wbar^n [j == jr],
 * evaluated as fma(c2, l_{j-1} + l_{j+1}, fma(k, l_j, -l2_j)) + wbar^n.
 * Outputs
 *   dg[n]  = dL/dfA[n] = c2 lambda^{n+1}_1 + wbar^n [jr == 0]   (dg[T] has only the direct term)
 *   *dc2   = dL/dc2    = sum_{n<T} sum_j lambda^{n+1}_j ((u^n_{j-1} + u^n_{j+1}) - 2 u^n_j)
 *   *abs_dc2 = the same sum of absolute values (conditioning of *dc2)
 * dL/da follows as dL/dc2 * 2 c2 / a.  The forward levels needed by the
 * backward sweep are recomputed segment by segment from checkpoints stored
 * every C = ceil(sqrt(T+1)) levels.
 */
int oracle_adjoint(int64_t nx, int64_t T, double c2, double k, const double* fA, const double* fB,
                   int64_t jr, const double* wbar, double* dg, double* dc2, double* abs_dc2)
{
    if (nx < 3 || T < 0 || jr < 0 || jr >= nx) return 1;
    int64_t C = (int64_t)ceil(sqrt((double)(T + 1)));
    int64_t nseg = (T + C - 1) / C; /* segments cover levels 0..T-1 */
    if (nseg < 1) nseg = 1;
    double* ck_u = (double*)malloc(sizeof(double) * nx * nseg);
    double* ck_p = (double*)malloc(sizeof(double) * nx * nseg);
    double* seg = (double*)malloc(sizeof(double) * nx * C);
    double* u = (double*)malloc(sizeof(double) * nx);
    double* up = (double*)malloc(sizeof(double) * nx);
    double* un = (double*)malloc(sizeof(double) * nx);
    double* l1 = (double*)calloc(nx, sizeof(double));
    double* l2 = (double*)calloc(nx, sizeof(double));
    double* ln = (double*)calloc(nx, sizeof(double));
    if (!ck_u || !ck_p || !seg || !u || !up || !un || !l1 || !l2 || !ln) {
        free(ck_u); free(ck_p); free(seg); free(u); free(up); free(un); free(l1); free(l2); free(ln);
        return 2;
    }
    /* forward sweep with checkpoints of (u^{mC}, u^{mC-1}) */
    for (int64_t j = 0; j < nx; ++j) u[j] = 0.0;
    u[0] = fA[0];
    u[nx - 1] = fB[0];
    memcpy(up, u, sizeof(double) * nx);
    for (int64_t n = 0; n < T; ++n) {
        if (n % C == 0) {
            memcpy(ck_u + (n / C) * nx, u, sizeof(double) * nx);
            memcpy(ck_p + (n / C) * nx, up, sizeof(double) * nx);
        }
        for (int64_t j = 1; j < nx - 1; ++j) un[j] = fma(c2, u[j - 1] + u[j + 1], fma(k, u[j], -up[j]));
        un[0] = fA[n + 1];
        un[nx - 1] = fB[n + 1];
        double* t = up; up = u; u = un; un = t;
    }
    /* backward sweep */
    double acc = 0.0, acc_abs = 0.0;
    dg[T] = (jr == 0) ? wbar[T] : 0.0;
    /* lambda^T (l1 holds lambda^{n+1}, l2 holds lambda^{n+2} at the top of the loop below) */
    for (int64_t j = 0; j < nx; ++j) { l1[j] = 0.0; l2[j] = 0.0; }
    if (jr > 0 && jr < nx - 1) l1[jr] = wbar[T];
    for (int64_t m = nseg - 1; m >= 0; --m) {
        int64_t n_lo = m * C;
        int64_t n_hi = (m + 1) * C < T ? (m + 1) * C : T; /* levels n_lo..n_hi-1 */
        /* recompute forward levels of the segment */
        memcpy(u, ck_u + m * nx, sizeof(double) * nx);
        memcpy(up, ck_p + m * nx, sizeof(double) * nx);
        for (int64_t n = n_lo; n < n_hi; ++n) {
            memcpy(seg + (n - n_lo) * nx, u, sizeof(double) * nx);
            for (int64_t j = 1; j < nx - 1; ++j) un[j] = fma(c2, u[j - 1] + u[j + 1], fma(k, u[j], -up[j]));
            un[0] = fA[n + 1];
            un[nx - 1] = fB[n + 1];
            double* t = up; up = u; u = un; un = t;
        }
        for (int64_t n = n_hi - 1; n >= n_lo; --n) {
            const double* un_ = seg + (n - n_lo) * nx; /* u^n */
            /* here l1 = lambda^{n+1}, l2 = lambda^{n+2} */
            dg[n] = c2 * l1[1] + ((jr == 0) ? wbar[n] : 0.0);
            for (int64_t j = 1; j < nx - 1; ++j) {
                double term = l1[j] * ((un_[j - 1] + un_[j + 1]) - 2.0 * un_[j]);
                acc += term;
                acc_abs += fabs(term);
            }
            if (n == 0) break; /* lambda^0 is not needed */
            ln[0] = 0.0;
            ln[nx - 1] = 0.0;
            for (int64_t j = 1; j < nx - 1; ++j) {
                double left = (j - 1 >= 1) ? l1[j - 1] : 0.0;
                double right = (j + 1 <= nx - 2) ? l1[j + 1] : 0.0;
                double v = fma(c2, left + right, fma(k, l1[j], -l2[j]));
                if (j == jr) v = v + wbar[n];
                ln[j] = v;
            }
            double* t = l2; l2 = l1; l1 = ln; ln = t;
        }
    }
    *dc2 = acc;
    if (abs_dc2) *abs_dc2 = acc_abs;
    free(ck_u); free(ck_p); free(seg); free(u); free(up); free(un); free(l1); free(l2); free(ln);
    return 0;
}
