/*
 * Body of the oracle's leapfrog and serial-RSWR routines, written once for a
 * floating type REAL and included twice by rswr_oracle.c (REAL = double and
 * REAL = float).  TEST INFRASTRUCTURE: see the header of rswr_oracle.c.
 *
 * Required macros: REAL, FMA (correctly rounded fused multiply-add for REAL),
 * NAME(x) (appends the precision suffix to a function name).
 *
 * Notation (paper Sec. 2.1): u(x,t) solves u_tt = a^2 u_xx on [X_A, X_B],
 * zero initial data, Dirichlet u(X_A,t) = f_A(t), u(X_B,t) = f_B(t).
 * Grid x_j = X_A + j dx, j = 0..nx-1; level n is t = n dt.
 *
 * The discretisation is the second-order central leapfrog (the paper fixes
 * none).  Two fixed operation orders are defined:
 *   form 0 ("canonical"):  u^{n+1}_j = fma(c2, u^n_{j-1} + u^n_{j+1},
 *                                         fma(k, u^n_j, -u^{n-1}_j)),  k = 2 - 2 c2
 *   form 1 ("increment"):  lap = (u_{j-1} - u_j) + (u_{j+1} - u_j)
 *                          v^{n+1}_j = fma(c2, lap, v^n_j)
 *                          u^{n+1}_j = u^n_j + v^{n+1}_j          (v^n = u^n - u^{n-1})
 * A state is a pair (q0, q1): form 0 holds (u^n, u^{n-1}); form 1 holds (u^n, v^n).
 */

/* One interior update of point j from the state (u, w) where w is u^{n-1}
 * (form 0) or v^n (form 1).  uL/uR are the neighbour values actually used
 * (true neighbours, or a ghost value at a guessed boundary). */
static inline void NAME(point_update)(int form, REAL c2, REAL k, REAL uL, REAL uC, REAL uR,
                                      REAL w, REAL* u_new, REAL* w_new)
{
    if (form == 0) {
        REAL s = uL + uR;
        REAL t = FMA(k, uC, -w);
        *u_new = FMA(c2, s, t);
        *w_new = uC; /* new "previous level" */
    } else {
        REAL lap = (uL - uC) + (uR - uC);
        REAL v = FMA(c2, lap, w);
        *u_new = uC + v;
        *w_new = v;
    }
}

/* Second state component at a Dirichlet node when the node moves from the
 * sample f_old to f_new: form 0 keeps the old value, form 1 the increment. */
static inline REAL NAME(dirichlet_w)(int form, REAL f_old, REAL f_new)
{
    return form == 0 ? f_old : (REAL)(f_new - f_old);
}

/* Level-0 state (paper Sec. 2.1: u(x,0) = 0, u_t(x,0) = 0, unless an initial
 * state is supplied).  Boundary nodes always take the Dirichlet samples at
 * t = 0; the second component at the boundary is "at rest". */
static void NAME(init_state)(int form, int64_t nx, const REAL* fA, const REAL* fB,
                             const REAL* q0, const REAL* q1, REAL* u, REAL* w)
{
    for (int64_t j = 0; j < nx; ++j) {
        u[j] = q0 ? q0[j] : (REAL)0;
    }
    u[0] = fA[0];
    u[nx - 1] = fB[0];
    for (int64_t j = 0; j < nx; ++j) {
        if (q1) w[j] = q1[j];
        else w[j] = (form == 0) ? u[j] : (REAL)0;
    }
    w[0] = (form == 0) ? u[0] : (REAL)0;
    w[nx - 1] = (form == 0) ? u[nx - 1] : (REAL)0;
}

/* Interior point sources entering level n+1 (the paper's pulse sources,
 * Sec. 4; with one source, also the source term of the discrete adjoint):
 * source q adds src[q*(T+1) + n+1] at point src_j[q] when level n+1 is formed,
 * to the new value (form 0) or to the new increment before it is applied
 * (form 1), in the order q = 0, 1, ...  Only points in [lo, hi] that are not a
 * Dirichlet node are touched; u_old is level n (form 1 recomputes u = u_old + v). */
static void NAME(add_sources)(int form, int64_t nx, int64_t T, int64_t n, int64_t nsrc, const int64_t* src_j,
                              const REAL* src, int64_t lo, int64_t hi, const REAL* u_old, REAL* un, REAL* wn)
{
    for (int64_t q = 0; q < nsrc; ++q) {
        int64_t j = src_j[q];
        if (j <= 0 || j >= nx - 1 || j < lo || j > hi) continue;
        REAL s = src[q * (T + 1) + n + 1];
        if (form == 0) {
            un[j] = un[j] + s;
        } else {
            wn[j] = wn[j] + s;
            un[j] = u_old[j] + wn[j];
        }
    }
}

/* Value and flux probes of one level: rec[r*(T+1)+n] = u_j, flux = (u_{j+1}-u_{j-1})*inv2dx. */
static void NAME(record)(int64_t n, int64_t T, const REAL* u, int64_t nrec, const int64_t* rec_j,
                         REAL* rec, int64_t nflux, const int64_t* flux_j, REAL inv2dx, REAL* flux)
{
    for (int64_t r = 0; r < nrec; ++r) rec[r * (T + 1) + n] = u[rec_j[r]];
    for (int64_t r = 0; r < nflux; ++r) {
        int64_t j = flux_j[r];
        flux[r * (T + 1) + n] = (u[j + 1] - u[j - 1]) * inv2dx;
    }
}

/*
 * Monolithic ("true solution", paper Sec. 2.1, Definition "True Solution")
 * leapfrog over the whole undecomposed domain for T steps.
 * Outputs the final state pair and optional per-level probes (n = 0..T).
 */
int NAME(oracle_leapfrog)(int form, int64_t nx, int64_t T, REAL c2, REAL k,
                          const REAL* fA, const REAL* fB, const REAL* q0, const REAL* q1,
                          REAL* out0, REAL* out1,
                          int64_t nrec, const int64_t* rec_j, REAL* rec,
                          int64_t nflux, const int64_t* flux_j, REAL inv2dx, REAL* flux,
                          int64_t nsrc, const int64_t* src_j, const REAL* src)
{
    if (nx < 3 || T < 0 || (form != 0 && form != 1)) return 1;
    REAL* u = (REAL*)malloc(sizeof(REAL) * nx);
    REAL* w = (REAL*)malloc(sizeof(REAL) * nx);
    REAL* un = (REAL*)malloc(sizeof(REAL) * nx);
    REAL* wn = (REAL*)malloc(sizeof(REAL) * nx);
    if (!u || !w || !un || !wn) { free(u); free(w); free(un); free(wn); return 2; }
    NAME(init_state)(form, nx, fA, fB, q0, q1, u, w);
    NAME(record)(0, T, u, nrec, rec_j, rec, nflux, flux_j, inv2dx, flux);
    for (int64_t n = 0; n < T; ++n) {
#pragma omp parallel for schedule(static) num_threads(oracle_nthreads) if (oracle_nthreads > 1)
        for (int64_t j = 1; j < nx - 1; ++j)
            NAME(point_update)(form, c2, k, u[j - 1], u[j], u[j + 1], w[j], &un[j], &wn[j]);
        if (src && nsrc > 0) NAME(add_sources)(form, nx, T, n, nsrc, src_j, src, 1, nx - 2, u, un, wn);
        un[0] = fA[n + 1];
        wn[0] = NAME(dirichlet_w)(form, fA[n], fA[n + 1]);
        un[nx - 1] = fB[n + 1];
        wn[nx - 1] = NAME(dirichlet_w)(form, fB[n], fB[n + 1]);
        REAL* t;
        t = u; u = un; un = t;
        t = w; w = wn; wn = t;
        NAME(record)(n + 1, T, u, nrec, rec_j, rec, nflux, flux_j, inv2dx, flux);
    }
    memcpy(out0, u, sizeof(REAL) * nx);
    memcpy(out1, w, sizeof(REAL) * nx);
    free(u); free(w); free(un); free(wn);
    return 0;
}

/*
 * Serial RSWR with the select step taken as an index mask (paper Sec. 2.2-2.6
 * for N = 2, Sec. 3 for N > 2).
 *
 * Decomposition (Sec. 2.2, Sec. 3): cores [b_i, b_{i+1}-1] with
 * b_i = floor(i nx / N); the window (subdomain) Omega_i extends ceil(ov/2)
 * points left of its core and floor(ov/2) points right of it (clipped to the
 * domain), so neighbouring windows share exactly ov points.
 *
 * Each span of S <= floor(ov/2) steps (Waveform Time Span Theorem, Sec. 2.4,
 * taken on the discrete domain of dependence of one cell per step):
 *   predict (Sec. 2.3): every window restarts from the true state and is
 *       advanced S steps with a zero input flux at each input boundary (mirror
 *       ghost u_{L-1} := u_{L+1}, u_{R+1} := u_{R-1}) and the Dirichlet data at
 *       the outer boundary;
 *   select  (Sec. 2.4): after s steps only window points at least s points away
 *       from a guessed boundary are valid; for s <= S that includes the core;
 *   update  (Sec. 2.5): the valid cores, combined (Sec. 2.5, last equation,
 *       with each overlap point given to the subdomain whose core contains it),
 *       form the true state at the end of the span;
 *   redo    (Sec. 2.6): the next span restarts from that state.
 * The boundary output waveforms (Sec. 2.2 definitions) of every interface are
 * recorded: traces[((i*2)+0)*(T+1)+n] is the flux of Omega_i at the left end of
 * Omega_{i+1}; traces[((i*2)+1)*(T+1)+n] the flux of Omega_{i+1} at the right
 * end of Omega_i.  Level 0 is recorded from the initial state.
 */
int NAME(oracle_rswr_mask)(int form, int64_t nx, int64_t T, REAL c2, REAL k,
                           const REAL* fA, const REAL* fB, const REAL* q0, const REAL* q1,
                           int64_t N, int64_t ov, int64_t S, REAL* out0, REAL* out1,
                           REAL inv2dx, REAL* traces, int64_t nsrc, const int64_t* src_j, const REAL* src)
{
    if (nx < 3 || T < 0 || N < 1 || ov < 2 || S < 1 || (form != 0 && form != 1)) return 1;
    int64_t el = (ov + 1) / 2, er = ov / 2;
    REAL* u = (REAL*)malloc(sizeof(REAL) * nx);
    REAL* w = (REAL*)malloc(sizeof(REAL) * nx);
    REAL* nu = (REAL*)malloc(sizeof(REAL) * nx);
    REAL* nw = (REAL*)malloc(sizeof(REAL) * nx);
    REAL* pu = (REAL*)malloc(sizeof(REAL) * nx);  /* predictive solution of one window */
    REAL* pw = (REAL*)malloc(sizeof(REAL) * nx);
    REAL* qu = (REAL*)malloc(sizeof(REAL) * nx);
    REAL* qw = (REAL*)malloc(sizeof(REAL) * nx);
    if (!u || !w || !nu || !nw || !pu || !pw || !qu || !qw) {
        free(u); free(w); free(nu); free(nw); free(pu); free(pw); free(qu); free(qw);
        return 2;
    }
    NAME(init_state)(form, nx, fA, fB, q0, q1, u, w);

    /* level-0 output waveforms from the initial state */
    for (int64_t i = 0; i + 1 < N; ++i) {
        int64_t b1 = (i + 1) * nx / N;
        int64_t Lnext = b1 - el < 0 ? 0 : b1 - el;
        int64_t Rthis = b1 - 1 + er > nx - 1 ? nx - 1 : b1 - 1 + er;
        if (traces) {
            traces[(i * 2 + 0) * (T + 1)] = (u[Lnext + 1] - u[Lnext - 1]) * inv2dx;
            traces[(i * 2 + 1) * (T + 1)] = (u[Rthis + 1] - u[Rthis - 1]) * inv2dx;
        }
    }

    for (int64_t n0 = 0; n0 < T; n0 += S) {
        int64_t steps = (T - n0 < S) ? (T - n0) : S;
        for (int64_t i = 0; i < N; ++i) {
            int64_t b0 = i * nx / N, b1 = (i + 1) * nx / N;
            int64_t L = b0 - el < 0 ? 0 : b0 - el;
            int64_t R = b1 - 1 + er > nx - 1 ? nx - 1 : b1 - 1 + er;
            /* predict: the window starts from the true state (Sec. 2.3, Sec. 2.6) */
            for (int64_t j = L; j <= R; ++j) { pu[j] = u[j]; pw[j] = w[j]; }
            for (int64_t s = 0; s < steps; ++s) {
                int64_t n = n0 + s;
                for (int64_t j = L; j <= R; ++j) {
                    if (j == 0) {
                        qu[j] = fA[n + 1];
                        qw[j] = NAME(dirichlet_w)(form, fA[n], fA[n + 1]);
                    } else if (j == nx - 1) {
                        qu[j] = fB[n + 1];
                        qw[j] = NAME(dirichlet_w)(form, fB[n], fB[n + 1]);
                    } else {
                        /* zero input flux guess at an input boundary (Sec. 2.3) */
                        REAL uL = (j == L) ? pu[j + 1] : pu[j - 1];
                        REAL uR = (j == R) ? pu[j - 1] : pu[j + 1];
                        NAME(point_update)(form, c2, k, uL, pu[j], uR, pw[j], &qu[j], &qw[j]);
                    }
                }
                /* the sources inside the window, halo included (Sec. 4 pulse sources) */
                if (src && nsrc > 0) NAME(add_sources)(form, nx, T, n, nsrc, src_j, src, L, R, pu, qu, qw);
                for (int64_t j = L; j <= R; ++j) { pu[j] = qu[j]; pw[j] = qw[j]; }
                /* boundary output waveforms of this window (Sec. 2.2 definitions) */
                if (traces) {
                    if (i + 1 < N) {
                        int64_t Lnext = b1 - el < 0 ? 0 : b1 - el;
                        traces[(i * 2 + 0) * (T + 1) + n + 1] = (pu[Lnext + 1] - pu[Lnext - 1]) * inv2dx;
                    }
                    if (i > 0) {
                        int64_t Rprev = b0 - 1 + er > nx - 1 ? nx - 1 : b0 - 1 + er;
                        traces[((i - 1) * 2 + 1) * (T + 1) + n + 1] = (pu[Rprev + 1] - pu[Rprev - 1]) * inv2dx;
                    }
                }
            }
            /* select + update: keep only the core (Sec. 2.4, Sec. 2.5 combination) */
            for (int64_t j = b0; j < b1; ++j) { nu[j] = pu[j]; nw[j] = pw[j]; }
        }
        REAL* t;
        t = u; u = nu; nu = t;
        t = w; w = nw; nw = t;
    }
    memcpy(out0, u, sizeof(REAL) * nx);
    memcpy(out1, w, sizeof(REAL) * nx);
    free(u); free(w); free(nu); free(nw); free(pu); free(pw); free(qu); free(qw);
    return 0;
}
