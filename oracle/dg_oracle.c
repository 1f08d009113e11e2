/*
 * dg_oracle.c -- plain, slow, FP64 CPU reference of the modal Discontinuous
 * Galerkin right-hand side, SSP Runge-Kutta step, CFL time step, oscillation
 * sensor and positivity limiter of Cernetic, Springel, Guillet & Pakmor,
 * "High-order Discontinuous Galerkin hydrodynamics with sub-cell shock
 * capturing on GPUs" (arXiv 2208.11131).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py
 * use it.  It shares no code, header, table or constant with the CUDA path.
 *
 * Every quantity is computed the direct way the paper writes it: a state value
 * at a quadrature point is the full sum over all modes, the volume integral is
 * the full sum over all volume Gauss points (Eq. time_stepping_final, with the
 * prefactors re-derived from Eq. weight_evolution: 2^(1-d)/h_alpha for both
 * the volume and the surface term), the interface recovery builds the joint
 * coefficients q of Eq. basisprojection and evaluates them at the face.  No
 * sum factorisation, no collocation, no fusion.  Compile with
 * -ffp-contract=off so that the compiler does not fuse multiply-adds.
 *
 * Readings of the paper taken here (where it is garbled or silent):
 *  - basis: full tensor product of scaled Legendre polynomials
 *    Pt_l = sqrt(2l+1) P_l (Sec. 2.3 normalisation, int Pt_l Pt_m = 2 delta),
 *    so w_0 is the cell mean;
 *  - quadrature: n+1 Gauss-Legendre points per axis (Sec. 2.4);
 *  - recovery (Sec. 3.2, Eq. basisprojection): prefactor 1/2 in the K* unit
 *    coordinate, A+ uses Pt_m(2 f x - 1), the sum runs over all normal modes
 *    m = 0..n, the joint polynomial has normal degree n+1; f = 3/4 for n <= 2
 *    and f = 1 for n > 2;
 *  - Riemann solver: textbook HLLC (Toro) with Davis wave-speed estimates;
 *  - viscous tensor (Sec. 3.3): Pi = nu rho (grad v + grad v^T - 2/3 div v I);
 *    heat flux chi (gamma-1) rho grad u_int with chi = kappa;
 *  - artificial viscosity (Sec. 4.1): eps = av_scale * clip(alpha,0,1) * c_s * h / P,
 *    P = n+1, h = min_alpha h_alpha; face eps = mean of the two trace values;
 *    alpha source f_v max(0,-div v) + wiggle term - alpha/tau with
 *    tau = f_tau h / (P c_s); the wiggle term is one value per cell per step,
 *    f_w max(0, dlogS/dt) [S > s_onset/P^2], dlogS/dt being the difference of
 *    ln S between the starts of this and the previous step over the previous
 *    step's dt, with S floored at 1e-4 s_onset/P^2 (below the floor the sensor
 *    value is rounding noise of the higher modes, and the log of noise would
 *    make the wiggle source noise / dt);
 *  - sensor (Eq. discontinuity_sensor2): density modes with max(l_x,l_y,l_z)=n;
 *  - time step (Eq. timestep): maxima of c_s and |v| over the volume Gauss
 *    points of the state at the start of the step, h = min_alpha h_alpha;
 *  - SSP Runge-Kutta: P stages for P <= 3 (forward Euler, Heun, Shu-Osher
 *    RK3) and the 5-stage 4th-order scheme of Spiteri & Ruuth (2002) above;
 *  - positivity limiter (Sec. 4.2): applied to the state entering each step
 *    and after every stage, to the conserved fields' higher modes; rho_b =
 *    1e-6 mean rho, p_b = 1e-6 p(mean state); pressure pass halves the higher
 *    modes, at most 60 times;
 *  - outflow boundary: the ghost trace equals the interior trace, so the face
 *    flux is the physical flux of the interior trace and no dissipative flux
 *    crosses the boundary.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXN 7
#define OR_MAXQ (OR_MAXN + 1)
#define OR_MAXF 7

/* status codes (shared meaning with the test suite only) */
#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENONPHYS 4

typedef struct {
    int dim, n;
    int N[3];
    double lo[3], hi[3];
    int bc[3]; /* 0 periodic, 1 outflow */
    double gamma, nu, kappa;
    int av_on;
    double av_scale, f_v, f_tau, f_w, s_onset;
    int positivity_on;
    double cfl;
    int rk_stages; /* 0: automatic choice from the order */
    /* turbulence driving (Sec. 7.1, "Driving"): amplitude of the |k| = 1 modes, OU correlation
     * time t_s, update interval, generator seed */
    int forcing_on;
    double force_amp, force_ts, force_dt;
    unsigned long long force_seed;
    /* passive tracer (Sec. 3.4): conserved field rho c after the energy, diffusivity eta */
    int tracer_on;
    double eta;
    /* basis (Sec. 2.3): 0 full tensor product (every l_a <= n), 1 the paper's total-degree set
     * (l_x + l_y + l_z <= n) */
    int basis;
    /* floor of the oscillation sensor inside the logarithm of the wiggle source, as a fraction
     * of the onset threshold s_onset/P^2 (1e-4: the reading of Sec. 4.1 used throughout) */
    double s_floor;
} or_cfg;

/* ------------------------------------------------------------------ */
/* Legendre polynomials and Gauss-Legendre quadrature (Sec. 2.3, 2.4)  */
/* ------------------------------------------------------------------ */

static double leg(int l, double x)
{
    double p0 = 1.0, p1 = x;
    if (l == 0) return 1.0;
    for (int k = 1; k < l; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

/* derivative through P'_{k+1} = P'_{k-1} + (2k+1) P_k */
static double dleg(int l, double x)
{
    double d[OR_MAXQ + 3];
    d[0] = 0.0;
    if (l == 0) return 0.0;
    d[1] = 1.0;
    for (int k = 1; k < l; ++k) d[k + 1] = d[k - 1] + (2.0 * k + 1.0) * leg(k, x);
    return d[l];
}

/* scaled Legendre polynomial, int_{-1}^{1} Pt_l Pt_m = 2 delta_lm */
double or_pt(int l, double x) { return sqrt(2.0 * l + 1.0) * leg(l, x); }
double or_dpt(int l, double x) { return sqrt(2.0 * l + 1.0) * dleg(l, x); }

/* q-point Gauss-Legendre rule on [-1,1], nodes ascending */
int or_gauss(int q, double *x, double *w)
{
    if (q < 1 || q > 64) return OR_EINVAL;
    for (int i = 0; i < q; ++i) {
        long double z = cosl(3.14159265358979323846264338327950288L * (i + 0.75L) / (q + 0.5L));
        long double pp = 0.0L;
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1.0L, p1 = z;
            if (q == 1) { p1 = z; p0 = 1.0L; }
            for (int k = 1; k < q; ++k) {
                long double p2 = ((2.0L * k + 1.0L) * z * p1 - k * p0) / (k + 1.0L);
                p0 = p1;
                p1 = p2;
            }
            /* p1 = P_q(z), p0 = P_{q-1}(z) */
            pp = q * (z * p1 - p0) / (z * z - 1.0L);
            long double dz = p1 / pp;
            z -= dz;
            if (fabsl(dz) < 1e-30L) break;
        }
        {
            long double p0 = 1.0L, p1 = z;
            for (int k = 1; k < q; ++k) {
                long double p2 = ((2.0L * k + 1.0L) * z * p1 - k * p0) / (k + 1.0L);
                p0 = p1;
                p1 = p2;
            }
            pp = q * (z * p1 - p0) / (z * z - 1.0L);
        }
        x[q - 1 - i] = (double)z;
        w[q - 1 - i] = (double)(2.0L / ((1.0L - z * z) * pp * pp));
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Tables of the direct (non-factorised) scheme                          */
/* ------------------------------------------------------------------ */

typedef struct {
    int d, n, Q, M, NQ, NQF, MT;
    double xg[OR_MAXQ], wg[OR_MAXQ];
    double *phi;   /* [NQ][M]       phi_l(xi_j) at volume points      */
    double *dphi;  /* [d][NQ][M]    d phi_l / d xi_alpha              */
    double *G;     /* [NQ]          tensor Gauss weight               */
    double *phif;  /* [d][2][NQF][M] phi_l on face side s (0:-1, 1:+1) */
    double *GF;    /* [NQF]         face Gauss weight                 */
    double *phit;  /* [d][NQF][MT]  transverse basis at face points    */
    double *dphit; /* [d][d-1][NQF][MT] transverse derivatives          */
    double f;      /* recovery overlap fraction                        */
    double Am[OR_MAXQ][OR_MAXQ + 1], Ap[OR_MAXQ][OR_MAXQ + 1];
    double P0[OR_MAXQ + 1], dP0[OR_MAXQ + 1];
} or_tab;

static void unflat(int idx, int base, int d, int *out)
{
    for (int a = 0; a < d; ++a) {
        out[a] = idx % base;
        idx /= base;
    }
}

static int flat(const int *idx, int base, int d)
{
    int r = 0;
    for (int a = d - 1; a >= 0; --a) r = r * base + idx[a];
    return r;
}

#define OR_MAXM (OR_MAXQ * OR_MAXQ * OR_MAXQ)

/* modes of the basis (Sec. 2.3): products Pt_lx Pt_ly Pt_lz with every l_a <= n (basis 0) or with
 * l_x + l_y + l_z <= n (basis 1, the paper's truncation), in tensor order (x fastest);
 * exps[l] = (l_x, l_y, l_z), mode_of[tensor index] = l or -1 if absent; returns the count */
static int mode_list(int d, int n, int basis, int (*exps)[3], int *mode_of)
{
    int Q = n + 1, T = 1, M = 0;
    for (int a = 0; a < d; ++a) T *= Q;
    for (int t = 0; t < T; ++t) {
        int ll[3] = {0, 0, 0};
        unflat(t, Q, d, ll);
        int sum = ll[0] + ll[1] + ll[2];
        if (basis == 1 && sum > n) {
            mode_of[t] = -1;
            continue;
        }
        for (int a = 0; a < 3; ++a) exps[M][a] = ll[a];
        mode_of[t] = M++;
    }
    return M;
}

int or_num_modes(int d, int n, int basis)
{
    int exps[OR_MAXM][3], mode_of[OR_MAXM];
    if (d < 2 || d > 3 || n < 0 || n > OR_MAXN) return -1;
    return mode_list(d, n, basis, exps, mode_of);
}

/* the transverse axes of a face normal to `ax`, in increasing order */
static void transverse_axes(int d, int ax, int *ta)
{
    int k = 0;
    for (int b = 0; b < d; ++b)
        if (b != ax) ta[k++] = b;
}

/* A-/A+ overlap integrals of Eq. basisprojection, by exact Gauss quadrature */
int or_recovery_matrices(int n, double f, double *Am, double *Ap)
{
    double x[OR_MAXQ + 4], w[OR_MAXQ + 4];
    int q = n + 3;
    if (n < 0 || n > OR_MAXN) return OR_EINVAL;
    or_gauss(q, x, w);
    for (int m = 0; m <= n; ++m)
        for (int l = 0; l <= n + 1; ++l) {
            double sm = 0.0, sp = 0.0;
            for (int j = 0; j < q; ++j) {
                double xm = -0.5 + 0.5 * x[j]; /* [-1,0] */
                double xp = 0.5 + 0.5 * x[j];  /* [0,1]  */
                sm += 0.5 * w[j] * or_pt(m, 2.0 * f * xm + 1.0) * or_pt(l, xm);
                sp += 0.5 * w[j] * or_pt(m, 2.0 * f * xp - 1.0) * or_pt(l, xp);
            }
            Am[m * (n + 2) + l] = sm;
            Ap[m * (n + 2) + l] = sp;
        }
    return OR_OK;
}

double or_overlap_fraction(int n) { return n <= 2 ? 0.75 : 1.0; }

static int tab_init(or_tab *T, int d, int n, int M_, const int (*exps)[3])
{
    int Q = n + 1;
    T->d = d;
    T->n = n;
    T->Q = Q;
    T->M = M_;
    T->NQ = 1;
    for (int a = 0; a < d; ++a) T->NQ *= Q;
    T->NQF = T->NQ / Q;
    T->MT = T->NQF;
    or_gauss(Q, T->xg, T->wg);
    int M = T->M, NQ = T->NQ, NQF = T->NQF, MT = T->MT;
    T->phi = malloc(sizeof(double) * NQ * M);
    T->dphi = malloc(sizeof(double) * d * NQ * M);
    T->G = malloc(sizeof(double) * NQ);
    T->phif = malloc(sizeof(double) * d * 2 * NQF * M);
    T->GF = malloc(sizeof(double) * NQF);
    T->phit = malloc(sizeof(double) * d * NQF * MT);
    T->dphit = malloc(sizeof(double) * d * (d - 1 > 0 ? d - 1 : 1) * NQF * MT);
    if (!T->phi || !T->dphi || !T->G || !T->phif || !T->GF || !T->phit || !T->dphit) return OR_EINVAL;

    for (int j = 0; j < NQ; ++j) {
        int jj[3];
        unflat(j, Q, d, jj);
        double g = 1.0;
        for (int a = 0; a < d; ++a) g *= T->wg[jj[a]];
        T->G[j] = g;
        for (int l = 0; l < M; ++l) {
            const int *ll = exps[l];
            double v = 1.0;
            for (int a = 0; a < d; ++a) v *= or_pt(ll[a], T->xg[jj[a]]);
            T->phi[j * M + l] = v;
            for (int b = 0; b < d; ++b) {
                double dv = 1.0;
                for (int a = 0; a < d; ++a)
                    dv *= (a == b) ? or_dpt(ll[a], T->xg[jj[a]]) : or_pt(ll[a], T->xg[jj[a]]);
                T->dphi[(b * NQ + j) * M + l] = dv;
            }
        }
    }
    for (int k = 0; k < NQF; ++k) {
        int kk[3] = {0, 0, 0};
        unflat(k, Q, d - 1, kk);
        double g = 1.0;
        for (int a = 0; a < d - 1; ++a) g *= T->wg[kk[a]];
        T->GF[k] = g;
    }
    for (int ax = 0; ax < d; ++ax) {
        int ta[2];
        transverse_axes(d, ax, ta);
        for (int s = 0; s < 2; ++s)
            for (int k = 0; k < NQF; ++k) {
                int kk[3] = {0, 0, 0};
                unflat(k, Q, d - 1, kk);
                double xi[3];
                xi[ax] = s ? 1.0 : -1.0;
                for (int a = 0; a < d - 1; ++a) xi[ta[a]] = T->xg[kk[a]];
                for (int l = 0; l < M; ++l) {
                    const int *ll = exps[l];
                    double v = 1.0;
                    for (int a = 0; a < d; ++a) v *= or_pt(ll[a], xi[a]);
                    T->phif[((ax * 2 + s) * NQF + k) * M + l] = v;
                }
            }
        for (int k = 0; k < NQF; ++k) {
            int kk[3] = {0, 0, 0};
            unflat(k, Q, d - 1, kk);
            for (int t = 0; t < MT; ++t) {
                int tt[3] = {0, 0, 0};
                unflat(t, Q, d - 1, tt);
                double v = 1.0;
                for (int a = 0; a < d - 1; ++a) v *= or_pt(tt[a], T->xg[kk[a]]);
                T->phit[(ax * NQF + k) * MT + t] = v;
                for (int b = 0; b < d - 1; ++b) {
                    double dv = 1.0;
                    for (int a = 0; a < d - 1; ++a)
                        dv *= (a == b) ? or_dpt(tt[a], T->xg[kk[a]]) : or_pt(tt[a], T->xg[kk[a]]);
                    T->dphit[((ax * (d - 1) + b) * NQF + k) * MT + t] = dv;
                }
            }
        }
    }
    T->f = or_overlap_fraction(n);
    {
        double Am[OR_MAXQ * (OR_MAXQ + 1)], Ap[OR_MAXQ * (OR_MAXQ + 1)];
        or_recovery_matrices(n, T->f, Am, Ap);
        for (int m = 0; m <= n; ++m)
            for (int l = 0; l <= n + 1; ++l) {
                T->Am[m][l] = Am[m * (n + 2) + l];
                T->Ap[m][l] = Ap[m * (n + 2) + l];
            }
    }
    for (int l = 0; l <= n + 1; ++l) {
        T->P0[l] = or_pt(l, 0.0);
        T->dP0[l] = or_dpt(l, 0.0);
    }
    return OR_OK;
}

static void tab_free(or_tab *T)
{
    free(T->phi);
    free(T->dphi);
    free(T->G);
    free(T->phif);
    free(T->GF);
    free(T->phit);
    free(T->dphit);
}

/* ------------------------------------------------------------------ */
/* Pointwise physics (Sec. 2.1, 3.3, 4.1)                               */
/* ------------------------------------------------------------------ */

typedef struct {
    double rho, v[3], p, cs, e;
} or_prim;

/* returns nonzero for a non-physical state (rho <= 0 or p <= 0) */
static int to_prim(const double *u, int d, double g, or_prim *P)
{
    P->rho = u[0];
    P->e = u[d + 1];
    double v2 = 0.0;
    for (int a = 0; a < 3; ++a) P->v[a] = 0.0;
    if (!(P->rho > 0.0)) {
        P->p = 0.0;
        P->cs = 0.0;
        return 1;
    }
    for (int a = 0; a < d; ++a) {
        P->v[a] = u[1 + a] / P->rho;
        v2 += P->v[a] * P->v[a];
    }
    P->p = (g - 1.0) * (P->e - 0.5 * P->rho * v2);
    if (!(P->p > 0.0)) {
        P->cs = 0.0;
        return 1;
    }
    P->cs = sqrt(g * P->p / P->rho);
    return 0;
}

/* Euler flux along axis ax, Eq. flux_matrix; with a tracer (tr = 1) its row c rho v_ax (Sec. 3.4) */
static void euler_flux_tr(const double *u, const or_prim *P, int d, int tr, int ax, double *F)
{
    double vn = P->v[ax];
    F[0] = u[0] * vn;
    for (int b = 0; b < d; ++b) F[1 + b] = u[1 + b] * vn + (b == ax ? P->p : 0.0);
    F[d + 1] = (P->e + P->p) * vn;
    if (tr) F[d + 2] = u[d + 2] * vn;
}


/* HLLC flux along axis ax (Toro), Davis wave-speed estimates; a passive tracer (tr = 1) is carried
 * in the star states with the concentration of its side, c_K rho*_K */
static int hllc_tr(int d, int tr, int ax, double g, const double *uL, const double *uR, double *F)
{
    or_prim L, R;
    int bad = to_prim(uL, d, g, &L) | to_prim(uR, d, g, &R);
    int nf = d + 2 + tr;
    double vL = L.v[ax], vR = R.v[ax];
    double SL = fmin(vL - L.cs, vR - R.cs);
    double SR = fmax(vL + L.cs, vR + R.cs);
    double FL[OR_MAXF], FR[OR_MAXF];
    euler_flux_tr(uL, &L, d, tr, ax, FL);
    euler_flux_tr(uR, &R, d, tr, ax, FR);
    if (SL >= 0.0) {
        for (int f = 0; f < nf; ++f) F[f] = FL[f];
        return bad;
    }
    double num = R.p - L.p + L.rho * vL * (SL - vL) - R.rho * vR * (SR - vR);
    double den = L.rho * (SL - vL) - R.rho * (SR - vR);
    double Ss = num / den;
    const double *uK;
    const or_prim *K;
    const double *FK;
    double SK;
    if (Ss >= 0.0) {
        uK = uL; K = &L; FK = FL; SK = SL;
    } else if (SR >= 0.0) {
        uK = uR; K = &R; FK = FR; SK = SR;
    } else {
        for (int f = 0; f < nf; ++f) F[f] = FR[f];
        return bad;
    }
    double vK = K->v[ax];
    double fac = K->rho * (SK - vK) / (SK - Ss);
    double us[OR_MAXF];
    us[0] = fac;
    for (int b = 0; b < d; ++b) us[1 + b] = fac * (b == ax ? Ss : K->v[b]);
    us[d + 1] = fac * (K->e / K->rho + (Ss - vK) * (Ss + K->p / (K->rho * (SK - vK))));
    if (tr) us[d + 2] = fac * (uK[d + 2] / K->rho);
    for (int f = 0; f < nf; ++f) F[f] = FK[f] + SK * (us[f] - uK[f]);
    return bad;
}

int or_hllc(int d, int ax, double g, const double *uL, const double *uR, double *F)
{
    return hllc_tr(d, 0, ax, g, uL, uR, F);
}

int or_hllc_tracer(int d, int ax, double g, const double *uL, const double *uR, double *F)
{
    return hllc_tr(d, 1, ax, g, uL, uR, F);
}

/* Navier-Stokes flux along axis ax from the state u and its physical
 * gradient grad[beta][field] (Sec. 3.3); with a tracer (tr = 1) its diffusion row
 * eta rho d_ax c = eta (d_ax (rho c) - c d_ax rho) (Sec. 3.4).  Returns nonzero if rho <= 0. */
static int ns_flux_tr(int d, int tr, int ax, double g, double nu, double kappa, double eta, const double *u,
                      const double *grad, double *F)
{
    int nf = d + 2 + tr;
    double rho = u[0];
    if (!(rho > 0.0)) return 1;
    double v[3] = {0, 0, 0};
    for (int b = 0; b < d; ++b) v[b] = u[1 + b] / rho;
    double dv[3][3];
    for (int be = 0; be < d; ++be)
        for (int b = 0; b < d; ++b) dv[be][b] = (grad[be * nf + 1 + b] - v[b] * grad[be * nf + 0]) / rho;
    double div = 0.0;
    for (int b = 0; b < d; ++b) div += dv[b][b];
    double Pi[3];
    for (int b = 0; b < d; ++b)
        Pi[b] = nu * rho * (dv[ax][b] + dv[b][ax] - (b == ax ? 2.0 / 3.0 * div : 0.0));
    double E = u[d + 1] / rho;
    double duint = (grad[ax * nf + d + 1] - E * grad[ax * nf + 0]) / rho;
    for (int b = 0; b < d; ++b) duint -= v[b] * dv[ax][b];
    F[0] = 0.0;
    double work = 0.0;
    for (int b = 0; b < d; ++b) {
        F[1 + b] = Pi[b];
        work += v[b] * Pi[b];
    }
    F[d + 1] = work + kappa * (g - 1.0) * rho * duint;
    if (tr) F[d + 2] = eta * (grad[ax * nf + d + 2] - (u[d + 2] / rho) * grad[ax * nf + 0]);
    return 0;
}

int or_ns_flux(int d, int ax, double g, double nu, double kappa, const double *u, const double *grad, double *F)
{
    return ns_flux_tr(d, 0, ax, g, nu, kappa, 0.0, u, grad, F);
}

static double clip01(double a) { return a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a); }

/* ------------------------------------------------------------------ */
/* Grid helpers                                                          */
/* ------------------------------------------------------------------ */

typedef struct {
    int d, n, Q, M, NF, FT, IA, TR;
    long ncell;
    int N[3];
    double h[3], hmin;
    int P;
    int need_grad;
    int diss; /* physical diffusive fluxes: NS (nu, kappa) and/or tracer diffusion (eta) */
    int basis;
    int exps[OR_MAXM][3]; /* exponents of mode l */
    int mode_of[OR_MAXM]; /* mode of a tensor index, -1 if not in the basis */
} or_geo;

static void geo_init(or_geo *g, const or_cfg *c)
{
    g->d = c->dim;
    g->n = c->n;
    g->Q = c->n + 1;
    g->basis = c->basis;
    g->ncell = 1;
    for (int a = 0; a < 3; ++a) g->N[a] = 1;
    g->hmin = 1e300;
    for (int a = 0; a < c->dim; ++a) {
        g->N[a] = c->N[a];
        g->ncell *= c->N[a];
        g->h[a] = (c->hi[a] - c->lo[a]) / c->N[a];
        if (g->h[a] < g->hmin) g->hmin = g->h[a];
    }
    g->TR = c->tracer_on ? 1 : 0;
    g->NF = c->dim + 2 + g->TR;
    g->FT = g->NF + (c->av_on ? 1 : 0);
    g->IA = g->NF;
    g->P = c->n + 1;
    g->diss = c->nu > 0.0 || c->kappa > 0.0 || (g->TR && c->eta > 0.0);
    g->need_grad = c->av_on || g->diss;
    g->M = mode_list(c->dim, c->n, c->basis, g->exps, g->mode_of);
}

static long cell_index(const or_geo *g, const int *ci)
{
    long r = 0;
    for (int a = g->d - 1; a >= 0; --a) r = r * g->N[a] + ci[a];
    return r;
}

static void cell_coords(const or_geo *g, long K, int *ci)
{
    for (int a = 0; a < g->d; ++a) {
        ci[a] = (int)(K % g->N[a]);
        K /= g->N[a];
    }
}

#define W(w, g, f, K, l) ((w)[((long)(f) * (g)->ncell + (K)) * (g)->M + (l)])

static int check_cfg(const or_cfg *c)
{
    if (c->dim < 2 || c->dim > 3) return OR_EINVAL;
    if (c->n < 0 || c->n > OR_MAXN) return OR_EINVAL;
    for (int a = 0; a < c->dim; ++a)
        if (c->N[a] < 1 || !(c->hi[a] > c->lo[a])) return OR_EINVAL;
    if (!(c->gamma > 1.0)) return OR_EINVAL;
    if (c->forcing_on && (!(c->force_ts > 0.0) || !(c->force_dt > 0.0) || !(c->force_amp >= 0.0)))
        return OR_EINVAL;
    if (c->tracer_on && !(c->eta >= 0.0)) return OR_EINVAL;
    if (c->basis != 0 && c->basis != 1) return OR_EINVAL;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Turbulence driving (Sec. 7.1, "Driving")                              */
/* ------------------------------------------------------------------ */
/* The acceleration field is a sum of Fourier modes with wave numbers 2pi/L <= |k| <= 2 (2pi/L),
 * amplitude proportional to |k|^(-5/3), whose complex vector coefficients follow independent
 * Ornstein-Uhlenbeck processes (correlation time t_s, advanced exactly at update instants
 * j * force_dt) and are projected onto the plane normal to k (solenoidal driving, the
 * projection equation of Sec. 7.1).  A real field needs one mode of every +-k pair:
 *   s(x) = sum_m  Re(s_m) cos(K_m.(x-lo)) - Im(s_m) sin(K_m.(x-lo)),
 *   s_m = A |k_m|^(-5/3) P(K_m) (X_m + i Y_m),  P(K) = I - K K^T / |K|^2,
 * K_m,a = 2 pi k_m,a / L_a, |k_m| in units of 2 pi / L.  X_m, Y_m are unit-variance OU
 * vectors (d components each).  Forcing state: fst[0] = index of the last update applied
 * (-1: none yet), fst[1 + 6 m + q] = component q of (X_m, Y_m) (q = 0..2 real, 3..5 imaginary;
 * components beyond d stay zero).
 * Random numbers: the SplitMix64 generator (Steele, Lea & Flood 2014) used counter-based,
 * output i of seed s is mix(s + (i+1) * 0x9E3779B97F4A7C15), mapped to (0,1) with 53 bits,
 * and the Box-Muller transform (1958) of outputs 2c and 2c+1 for the normal draw of counter c;
 * counter of (update j, mode m, component q) is (16 j + m) * 6 + q. */

#define OR_FMODES 16 /* mode stride: the 3-D count; 2-D has 6 */
#define OR_FSTATE (1 + 6 * OR_FMODES)

static const double OR_PI = 3.14159265358979323846;

/* wave vectors with 1 <= |k|^2 <= 4 whose first non-zero component is positive,
 * in loop order kz (outer), ky, kx (inner); returns their count */
int or_forcing_modes(int d, int *k)
{
    int n = 0;
    int zr = d == 3 ? 2 : 0;
    for (int kz = -zr; kz <= zr; ++kz)
        for (int ky = -2; ky <= 2; ++ky)
            for (int kx = -2; kx <= 2; ++kx) {
                int k2 = kx * kx + ky * ky + kz * kz;
                if (k2 < 1 || k2 > 4) continue;
                int first = kx != 0 ? kx : (ky != 0 ? ky : kz);
                if (first < 0) continue;
                k[3 * n + 0] = kx;
                k[3 * n + 1] = ky;
                k[3 * n + 2] = kz;
                ++n;
            }
    return n;
}

static uint64_t splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double or_forcing_uniform(unsigned long long seed, unsigned long long i)
{
    return ((double)(splitmix64_at(seed, i) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

double or_forcing_normal(unsigned long long seed, unsigned long long c)
{
    double u1 = or_forcing_uniform(seed, 2 * c), u2 = or_forcing_uniform(seed, 2 * c + 1);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * OR_PI * u2);
}

/* apply every OU update due at time t (update j at time j * force_dt; j = 0 draws the
 * stationary initial state) */
int or_forcing_update(const or_cfg *c, double *fst, double t)
{
    if (check_cfg(c) || !c->forcing_on) return OR_EINVAL;
    int k[3 * OR_FMODES];
    int nm = or_forcing_modes(c->dim, k);
    double f = exp(-c->force_dt / c->force_ts), g = sqrt(1.0 - f * f);
    long j = (long)fst[0];
    if (fst[0] < 0.0) {
        j = 0;
        for (int m = 0; m < nm; ++m)
            for (int q = 0; q < 6; ++q)
                fst[1 + 6 * m + q] = (q % 3) < c->dim ? or_forcing_normal(c->force_seed, (uint64_t)m * 6 + q) : 0.0;
    }
    long count = 0;
    while ((double)(j + 1) * c->force_dt <= t) {
        if (++count > 10000000L) return OR_EINVAL;
        ++j;
        for (int m = 0; m < nm; ++m)
            for (int q = 0; q < 6; ++q) {
                if ((q % 3) >= c->dim) continue;
                double xi = or_forcing_normal(c->force_seed, ((uint64_t)j * OR_FMODES + m) * 6 + q);
                fst[1 + 6 * m + q] = f * fst[1 + 6 * m + q] + g * xi;
            }
    }
    fst[0] = (double)j;
    return OR_OK;
}

/* driving acceleration at physical points x[npts][d] -> s[npts][3] */
int or_forcing_eval(const or_cfg *c, const double *fst, int npts, const double *x, double *s)
{
    if (check_cfg(c)) return OR_EINVAL;
    int d = c->dim;
    int k[3 * OR_FMODES];
    int nm = or_forcing_modes(d, k);
    for (int i = 0; i < npts; ++i) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int m = 0; m < nm; ++m) {
            double K[3] = {0.0, 0.0, 0.0}, K2 = 0.0, kk = 0.0, ph = 0.0;
            for (int a = 0; a < d; ++a) {
                K[a] = 2.0 * OR_PI * k[3 * m + a] / (c->hi[a] - c->lo[a]);
                K2 += K[a] * K[a];
                kk += (double)k[3 * m + a] * k[3 * m + a];
                ph += K[a] * (x[i * d + a] - c->lo[a]);
            }
            double amp = c->force_amp * pow(sqrt(kk), -5.0 / 3.0);
            const double *X = fst + 1 + 6 * m, *Y = X + 3;
            double KX = 0.0, KY = 0.0;
            for (int a = 0; a < d; ++a) {
                KX += K[a] * X[a];
                KY += K[a] * Y[a];
            }
            double cs = cos(ph), sn = sin(ph);
            for (int a = 0; a < d; ++a) {
                double re = X[a] - K[a] * KX / K2, im = Y[a] - K[a] * KY / K2;
                acc[a] += amp * (re * cs - im * sn);
            }
        }
        for (int a = 0; a < 3; ++a) s[i * 3 + a] = acc[a];
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Right-hand side  dw/dt = L(w)   (Eq. weight_evolution)               */
/* ------------------------------------------------------------------ */

/* state at the points of one face of cell K: side s (0: xi_ax=-1, 1: +1) */
static void face_trace(const or_tab *T, const or_geo *g, const double *w, long K, int ax, int s, int k, int nfields,
                       double *u)
{
    const double *ph = T->phif + ((ax * 2 + s) * T->NQF + k) * T->M;
    for (int f = 0; f < nfields; ++f) {
        double acc = 0.0;
        for (int l = 0; l < g->M; ++l) acc += W(w, g, f, K, l) * ph[l];
        u[f] = acc;
    }
}

/* Interface recovery (Sec. 3.2): the joint coefficients q of
 * Eq. basisprojection for every conserved field, evaluated at the face points:
 * ut[k][f] (state) and gt[k][beta][f] (physical gradient). */
static void face_recovery(const or_tab *T, const or_geo *g, const double *w, long KL, long KR, int ax, double *ut,
                          double *gt)
{
    int d = g->d, n = g->n, Q = g->Q, NF = g->NF;
    int MT = T->MT, NQF = T->NQF;
    int ta[2];
    transverse_axes(d, ax, ta);
    double q[OR_MAXQ + 1][OR_MAXQ * OR_MAXQ];
    for (int f = 0; f < NF; ++f) {
        for (int la = 0; la <= n + 1; ++la)
            for (int t = 0; t < MT; ++t) {
                int tt[3] = {0, 0, 0};
                unflat(t, Q, d - 1, tt);
                double acc = 0.0;
                for (int m = 0; m <= n; ++m) {
                    int ll[3];
                    ll[ax] = m;
                    for (int a = 0; a < d - 1; ++a) ll[ta[a]] = tt[a];
                    int l = g->mode_of[flat(ll, Q, d)];
                    if (l < 0) continue; /* absent from the basis: zero weight */
                    acc += T->Am[m][la] * W(w, g, f, KL, l) + T->Ap[m][la] * W(w, g, f, KR, l);
                }
                q[la][t] = 0.5 * acc;
            }
        for (int k = 0; k < NQF; ++k) {
            const double *pt = T->phit + (ax * NQF + k) * MT;
            double val = 0.0, dn = 0.0;
            double dt[2] = {0.0, 0.0};
            for (int la = 0; la <= n + 1; ++la)
                for (int t = 0; t < MT; ++t) {
                    val += q[la][t] * T->P0[la] * pt[t];
                    dn += q[la][t] * T->dP0[la] * pt[t];
                    for (int b = 0; b < d - 1; ++b)
                        dt[b] += q[la][t] * T->P0[la] * T->dphit[((ax * (d - 1) + b) * NQF + k) * MT + t];
                }
            ut[k * NF + f] = val;
            gt[(k * 3 + ax) * NF + f] = dn / (T->f * g->h[ax]);
            for (int b = 0; b < d - 1; ++b) gt[(k * 3 + ta[b]) * NF + f] = dt[b] * 2.0 / g->h[ta[b]];
        }
    }
}

/* artificial-viscosity coefficient eps = av_scale * clip(alpha) * c_s * h / P */
static double av_eps(const or_cfg *c, const or_geo *g, double alpha, double cs)
{
    return c->av_scale * clip01(alpha) * cs * g->hmin / g->P;
}

/* numerical flux at every point of the face at position p along axis ax,
 * between the cells with coordinates (p-1) and p along ax; returns status */
static int face_flux(const or_cfg *c, const or_tab *T, const or_geo *g, const double *w, int ax, const int *cf, int p,
                     double *Fh /* [NQF][NF] */)
{
    int d = g->d, NF = g->NF, FT = g->FT, NQF = T->NQF;
    int status = OR_OK;
    int cl[3], cr[3];
    for (int a = 0; a < 3; ++a) cl[a] = cr[a] = cf[a];
    int Nax = g->N[ax];
    int left_out = 0, right_out = 0;
    if (c->bc[ax] == 0) {
        cl[ax] = (p - 1 + Nax) % Nax;
        cr[ax] = p % Nax;
    } else {
        cl[ax] = p - 1;
        cr[ax] = p;
        if (p == 0) left_out = 1;
        if (p == Nax) right_out = 1;
    }
    if (left_out || right_out) {
        long K = cell_index(g, left_out ? cr : cl);
        int s = left_out ? 0 : 1;
        for (int k = 0; k < NQF; ++k) {
            double u[OR_MAXF];
            or_prim P;
            face_trace(T, g, w, K, ax, s, k, NF, u);
            if (to_prim(u, d, c->gamma, &P)) status = OR_ENONPHYS;
            euler_flux_tr(u, &P, d, g->TR, ax, Fh + k * NF);
        }
        return status;
    }
    long KL = cell_index(g, cl), KR = cell_index(g, cr);
    double uL[OR_MAXQ * OR_MAXQ][OR_MAXF], uR[OR_MAXQ * OR_MAXQ][OR_MAXF];
    for (int k = 0; k < NQF; ++k) {
        face_trace(T, g, w, KL, ax, 1, k, FT, uL[k]);
        face_trace(T, g, w, KR, ax, 0, k, FT, uR[k]);
        if (hllc_tr(d, g->TR, ax, c->gamma, uL[k], uR[k], Fh + k * NF)) status = OR_ENONPHYS;
    }
    int ns = g->diss;
    if (!ns && !c->av_on) return status;
    double ut[OR_MAXQ * OR_MAXQ * OR_MAXF];
    double gt[OR_MAXQ * OR_MAXQ * 3 * OR_MAXF];
    memset(gt, 0, sizeof(gt));
    face_recovery(T, g, w, KL, KR, ax, ut, gt);
    for (int k = 0; k < NQF; ++k) {
        double Fd[OR_MAXF];
        for (int f = 0; f < NF; ++f) Fd[f] = 0.0;
        if (ns) {
            double grad[3 * OR_MAXF];
            for (int b = 0; b < d; ++b)
                for (int f = 0; f < NF; ++f) grad[b * NF + f] = gt[(k * 3 + b) * NF + f];
            if (ns_flux_tr(d, g->TR, ax, c->gamma, c->nu, c->kappa, c->eta, ut + k * NF, grad, Fd))
                status = OR_ENONPHYS;
        }
        if (c->av_on) {
            or_prim PL, PR;
            if (to_prim(uL[k], d, c->gamma, &PL) | to_prim(uR[k], d, c->gamma, &PR)) status = OR_ENONPHYS;
            double eps = 0.5 * (av_eps(c, g, uL[k][g->IA], PL.cs) + av_eps(c, g, uR[k][g->IA], PR.cs));
            for (int f = 0; f < NF; ++f) Fd[f] += eps * gt[(k * 3 + ax) * NF + f];
        }
        for (int f = 0; f < NF; ++f) Fh[k * NF + f] -= Fd[f];
    }
    return status;
}

/* number of face positions along ax for a given transverse cell row */
static int face_positions(const or_cfg *c, const or_geo *g, int ax) { return c->bc[ax] == 0 ? g->N[ax] : g->N[ax] + 1; }

/* right-hand side; with fst (forcing on) the driving source of Sec. 7.1 is added: rho s to the
 * momentum and rho s.v = s.(rho v) to the energy, Gauss-integrated like every volume term */
int or_rhs_forced(const or_cfg *c, const double *w, const double *wig, const double *fst, double *rhs)
{
    if (check_cfg(c)) return OR_EINVAL;
    or_geo g;
    geo_init(&g, c);
    or_tab T;
    if (tab_init(&T, g.d, g.n, g.M, (const int(*)[3])g.exps)) return OR_EINVAL;
    int d = g.d, M = g.M, NQ = T.NQ, NQF = T.NQF, NF = g.NF, FT = g.FT;
    int status = OR_OK;
    double two1d = ldexp(1.0, 1 - d), two_d = ldexp(1.0, -d);
    memset(rhs, 0, sizeof(double) * (size_t)FT * g.ncell * M);
    int ns = g.diss;

    /* volume integral and alpha source (per cell) */
#pragma omp parallel for schedule(static) reduction(| : status)
    for (long K = 0; K < g.ncell; ++K) {
        for (int j = 0; j < NQ; ++j) {
            double u[OR_MAXF], grad[3 * OR_MAXF];
            const double *ph = T.phi + j * M;
            for (int f = 0; f < FT; ++f) {
                double acc = 0.0;
                for (int l = 0; l < M; ++l) acc += W(w, &g, f, K, l) * ph[l];
                u[f] = acc;
            }
            if (g.need_grad)
                for (int b = 0; b < d; ++b) {
                    const double *dp = T.dphi + (b * NQ + j) * M;
                    for (int f = 0; f < NF; ++f) {
                        double acc = 0.0;
                        for (int l = 0; l < M; ++l) acc += W(w, &g, f, K, l) * dp[l];
                        grad[b * NF + f] = acc * 2.0 / g.h[b];
                    }
                }
            or_prim P;
            if (to_prim(u, d, c->gamma, &P)) status |= OR_ENONPHYS;
            double eps = c->av_on ? av_eps(c, &g, u[g.IA], P.cs) : 0.0;
            double Fx[3][OR_MAXF];
            for (int ax = 0; ax < d; ++ax) {
                euler_flux_tr(u, &P, d, g.TR, ax, Fx[ax]);
                if (ns) {
                    double Fn[OR_MAXF];
                    ns_flux_tr(d, g.TR, ax, c->gamma, c->nu, c->kappa, c->eta, u, grad, Fn);
                    for (int f = 0; f < NF; ++f) Fx[ax][f] -= Fn[f];
                }
                if (c->av_on)
                    for (int f = 0; f < NF; ++f) Fx[ax][f] -= eps * grad[ax * NF + f];
            }
            for (int ax = 0; ax < d; ++ax) {
                const double *dp = T.dphi + (ax * NQ + j) * M;
                double cax = two1d / g.h[ax] * T.G[j];
                for (int f = 0; f < NF; ++f)
                    for (int l = 0; l < M; ++l) W(rhs, &g, f, K, l) += cax * dp[l] * Fx[ax][f];
            }
            if (c->av_on) {
                double div = 0.0;
                for (int b = 0; b < d; ++b) div += (grad[b * NF + 1 + b] - P.v[b] * grad[b * NF + 0]) / u[0];
                double adot = c->f_v * fmax(0.0, -div) + (wig ? wig[K] : 0.0) -
                              u[g.IA] * g.P * P.cs / (c->f_tau * g.hmin);
                for (int l = 0; l < M; ++l) W(rhs, &g, g.IA, K, l) += two_d * T.G[j] * ph[l] * adot;
            }
            if (c->forcing_on && fst) {
                int ci[3], jj[3];
                cell_coords(&g, K, ci);
                unflat(j, T.Q, d, jj);
                double xp[3], sv[3];
                for (int a = 0; a < d; ++a) xp[a] = c->lo[a] + (ci[a] + 0.5 + 0.5 * T.xg[jj[a]]) * g.h[a];
                or_forcing_eval(c, fst, 1, xp, sv);
                double src[OR_MAXF] = {0.0};
                for (int a = 0; a < d; ++a) {
                    src[1 + a] = u[0] * sv[a];
                    src[d + 1] += sv[a] * u[1 + a];
                }
                for (int f = 1; f < d + 2; ++f)
                    for (int l = 0; l < M; ++l) W(rhs, &g, f, K, l) += two_d * T.G[j] * ph[l] * src[f];
            }
        }
    }

    /* face fluxes, stored per axis and face position */
    double *Fh[3] = {NULL, NULL, NULL};
    long nfaces[3];
    for (int ax = 0; ax < d; ++ax) {
        int np = face_positions(c, &g, ax);
        long ntr = g.ncell / g.N[ax];
        nfaces[ax] = (long)np * ntr;
        Fh[ax] = malloc(sizeof(double) * nfaces[ax] * NQF * NF);
        if (!Fh[ax]) status |= OR_EINVAL;
    }
    if (status & OR_EINVAL) goto done;
    for (int ax = 0; ax < d; ++ax) {
        int np = face_positions(c, &g, ax);
        long nf_ax = nfaces[ax];
#pragma omp parallel for schedule(static) reduction(| : status)
        for (long fi = 0; fi < nf_ax; ++fi) {
            /* face index = p + np * (transverse cell row), rows ordered like cells with N[ax]=1 */
            int p = (int)(fi % np);
            long row = fi / np;
            int cf[3] = {0, 0, 0};
            long r = row;
            for (int a = 0; a < d; ++a) {
                if (a == ax) continue;
                cf[a] = (int)(r % g.N[a]);
                r /= g.N[a];
            }
            status |= face_flux(c, &T, &g, w, ax, cf, p, Fh[ax] + fi * NQF * NF);
        }
    }
    /* lift the face fluxes into both adjacent cells, in a fixed order */
#pragma omp parallel for schedule(static)
    for (long K = 0; K < g.ncell; ++K) {
        int ci[3];
        cell_coords(&g, K, ci);
        for (int ax = 0; ax < d; ++ax) {
            int np = face_positions(c, &g, ax);
            long row = 0, mul = 1;
            for (int a = 0; a < d; ++a) {
                if (a == ax) continue;
                row += ci[a] * mul;
                mul *= g.N[a];
            }
            int pl = ci[ax], pr = ci[ax] + 1;
            if (c->bc[ax] == 0) pr %= g.N[ax];
            const double *FL = Fh[ax] + (pl + np * row) * NQF * NF;
            const double *FR = Fh[ax] + (pr + np * row) * NQF * NF;
            double cax = two1d / g.h[ax];
            for (int k = 0; k < NQF; ++k) {
                const double *phm = T.phif + ((ax * 2 + 0) * NQF + k) * M;
                const double *php = T.phif + ((ax * 2 + 1) * NQF + k) * M;
                for (int f = 0; f < NF; ++f)
                    for (int l = 0; l < M; ++l) {
                        W(rhs, &g, f, K, l) -= cax * T.GF[k] * php[l] * FR[k * NF + f];
                        W(rhs, &g, f, K, l) += cax * T.GF[k] * phm[l] * FL[k * NF + f];
                    }
            }
        }
    }
done:
    for (int ax = 0; ax < d; ++ax) free(Fh[ax]);
    tab_free(&T);
    return status;
}

/* ------------------------------------------------------------------ */
/* Time step (Eq. timestep), sensor (Eq. discontinuity_sensor2)          */
/* ------------------------------------------------------------------ */

int or_max_speeds(const or_cfg *c, const double *w, double *cmax, double *vmax)
{
    if (check_cfg(c)) return OR_EINVAL;
    or_geo g;
    geo_init(&g, c);
    or_tab T;
    if (tab_init(&T, g.d, g.n, g.M, (const int(*)[3])g.exps)) return OR_EINVAL;
    double cm = 0.0, vm = 0.0;
    int status = OR_OK;
#pragma omp parallel for schedule(static) reduction(max : cm, vm) reduction(| : status)
    for (long K = 0; K < g.ncell; ++K)
        for (int j = 0; j < T.NQ; ++j) {
            double u[OR_MAXF];
            for (int f = 0; f < g.NF; ++f) {
                double acc = 0.0;
                for (int l = 0; l < g.M; ++l) acc += W(w, &g, f, K, l) * T.phi[j * g.M + l];
                u[f] = acc;
            }
            or_prim P;
            if (to_prim(u, g.d, c->gamma, &P)) status |= OR_ENONPHYS;
            double v2 = 0.0;
            for (int a = 0; a < g.d; ++a) v2 += P.v[a] * P.v[a];
            cm = fmax(cm, P.cs);
            vm = fmax(vm, sqrt(v2));
        }
    *cmax = cm;
    *vmax = vm;
    tab_free(&T);
    return status;
}

int or_max_dt(const or_cfg *c, const double *w, double *dt)
{
    double cm, vm;
    int st = or_max_speeds(c, w, &cm, &vm);
    if (st == OR_EINVAL) return st;
    or_geo g;
    geo_init(&g, c);
    *dt = c->cfl * g.hmin / (2.0 * g.P * (cm + vm));
    return st;
}

int or_sensor(const or_cfg *c, const double *w, double *S)
{
    if (check_cfg(c)) return OR_EINVAL;
    or_geo g;
    geo_init(&g, c);
#pragma omp parallel for schedule(static)
    for (long K = 0; K < g.ncell; ++K) {
        double hi = 0.0, all = 0.0;
        for (int l = 0; l < g.M; ++l) {
            const int *ll = g.exps[l];
            /* the modes the degree-(n-1) basis lacks: some l_a = n (tensor), l_x+l_y+l_z = n (total) */
            int top = 0;
            if (g.basis == 1) {
                top = ll[0] + ll[1] + ll[2] == g.n;
            } else {
                for (int a = 0; a < g.d; ++a)
                    if (ll[a] == g.n) top = 1;
            }
            double v = W(w, &g, 0, K, l);
            all += v * v;
            if (top && g.n > 0) hi += v * v;
        }
        S[K] = all > 0.0 ? hi / all : 0.0;
    }
    return OR_OK;
}

/* per-step wiggle source of the artificial-viscosity field (Sec. 4.1) */
int or_wiggle(const or_cfg *c, const double *w, double *S_prev, double *wig, double dt_prev, long step)
{
    if (check_cfg(c)) return OR_EINVAL;
    or_geo g;
    geo_init(&g, c);
    double *S = malloc(sizeof(double) * g.ncell);
    if (!S) return OR_EINVAL;
    or_sensor(c, w, S);
    double s_on = c->s_onset / ((double)g.P * g.P);
    double s_floor = c->s_floor * s_on;
    for (long K = 0; K < g.ncell; ++K) {
        double dlog = 0.0;
        if (step > 0 && dt_prev > 0.0) dlog = (log(fmax(S[K], s_floor)) - log(fmax(S_prev[K], s_floor))) / dt_prev;
        wig[K] = (S[K] > s_on) ? c->f_w * fmax(0.0, dlog) : 0.0;
        S_prev[K] = S[K];
    }
    free(S);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Positivity limiter (Sec. 4.2)                                         */
/* ------------------------------------------------------------------ */

int or_positivity(const or_cfg *c, double *w)
{
    if (check_cfg(c)) return OR_EINVAL;
    or_geo g;
    geo_init(&g, c);
    or_tab T;
    if (tab_init(&T, g.d, g.n, g.M, (const int(*)[3])g.exps)) return OR_EINVAL;
    int d = g.d, M = g.M, NF = g.NF;
    int npts = T.NQ + 2 * d * T.NQF;
    int status = OR_OK;
#pragma omp parallel for schedule(static) reduction(| : status)
    for (long K = 0; K < g.ncell; ++K) {
        double um[OR_MAXF];
        for (int f = 0; f < NF; ++f) um[f] = W(w, &g, f, K, 0);
        or_prim Pm;
        if (to_prim(um, d, c->gamma, &Pm)) {
            status |= OR_ENONPHYS;
            continue;
        }
        double rb = 1e-6 * um[0], pb = 1e-6 * Pm.p;
        double rmin = 1e300;
        for (int i = 0; i < npts; ++i) {
            const double *ph = i < T.NQ ? T.phi + i * M : T.phif + (i - T.NQ) * M;
            double r = 0.0;
            for (int l = 0; l < M; ++l) r += W(w, &g, 0, K, l) * ph[l];
            rmin = fmin(rmin, r);
        }
        if (rmin < rb) {
            double th = (um[0] - rb) / (um[0] - rmin);
            for (int f = 0; f < NF; ++f)
                for (int l = 1; l < M; ++l) W(w, &g, f, K, l) *= th;
        }
        int it = 0;
        for (;;) {
            double pmin = 1e300;
            for (int i = 0; i < npts; ++i) {
                const double *ph = i < T.NQ ? T.phi + i * M : T.phif + (i - T.NQ) * M;
                double u[OR_MAXF];
                for (int f = 0; f < NF; ++f) {
                    double acc = 0.0;
                    for (int l = 0; l < M; ++l) acc += W(w, &g, f, K, l) * ph[l];
                    u[f] = acc;
                }
                double v2 = 0.0;
                for (int a = 0; a < d; ++a) v2 += u[1 + a] * u[1 + a];
                double p = (c->gamma - 1.0) * (u[d + 1] - 0.5 * v2 / u[0]);
                pmin = fmin(pmin, p);
            }
            if (pmin >= pb) break;
            if (it == 60) {
                status |= OR_ENONPHYS;
                break;
            }
            for (int f = 0; f < NF; ++f)
                for (int l = 1; l < M; ++l) W(w, &g, f, K, l) *= 0.5;
            ++it;
        }
    }
    tab_free(&T);
    return status;
}

/* ------------------------------------------------------------------ */
/* SSP Runge-Kutta step (Sec. 2.5), Shu-Osher form                       */
/* ------------------------------------------------------------------ */

/* stage count for a given order P = n+1 */
int or_rk_stages(int n) { return n + 1 <= 3 ? n + 1 : 5; }

/* Shu-Osher coefficients alpha[i][k], beta[i][k] for stage i = 1..s
 * (u_i = sum_k alpha_ik u_k + beta_ik dt L(u_k)), row-major 6x6. */
int or_rk_table(int s, double *alpha, double *beta)
{
    for (int i = 0; i < 36; ++i) alpha[i] = beta[i] = 0.0;
#define A_(i, k) alpha[(i) * 6 + (k)]
#define B_(i, k) beta[(i) * 6 + (k)]
    switch (s) {
    case 1:
        A_(1, 0) = 1.0; B_(1, 0) = 1.0;
        break;
    case 2: /* Heun, SSP(2,2) */
        A_(1, 0) = 1.0; B_(1, 0) = 1.0;
        A_(2, 0) = 0.5; A_(2, 1) = 0.5; B_(2, 1) = 0.5;
        break;
    case 3: /* Shu-Osher SSP(3,3) */
        A_(1, 0) = 1.0; B_(1, 0) = 1.0;
        A_(2, 0) = 0.75; A_(2, 1) = 0.25; B_(2, 1) = 0.25;
        A_(3, 0) = 1.0 / 3.0; A_(3, 2) = 2.0 / 3.0; B_(3, 2) = 2.0 / 3.0;
        break;
    case 5: /* Spiteri & Ruuth (2002) SSP(5,4) */
        A_(1, 0) = 1.0; B_(1, 0) = 0.391752226571890;
        A_(2, 0) = 0.444370493651235; A_(2, 1) = 0.555629506348765; B_(2, 1) = 0.368410593050371;
        A_(3, 0) = 0.620101851488403; A_(3, 2) = 0.379898148511597; B_(3, 2) = 0.251891774271694;
        A_(4, 0) = 0.178079954393132; A_(4, 3) = 0.821920045606868; B_(4, 3) = 0.544974750228521;
        A_(5, 2) = 0.517231671970585; A_(5, 3) = 0.096059710526147; B_(5, 3) = 0.063692468666290;
        A_(5, 4) = 0.386708617503269; B_(5, 4) = 0.226007483236906;
        break;
    default:
        return OR_EINVAL;
    }
#undef A_
#undef B_
    return OR_OK;
}

int or_rhs(const or_cfg *c, const double *w, const double *wig, double *rhs)
{
    if (c->forcing_on) return OR_EINVAL; /* the forcing state is an argument of or_rhs_forced */
    return or_rhs_forced(c, w, wig, NULL, rhs);
}

/* one SSP-RK step of size dt (dt <= 0: CFL time step of the current state).
 * w is advanced in place; S_prev/wig are the per-cell sensor scalars;
 * scal = {dt_prev, step, t} is updated; dt_used receives the step size.
 * With forcing on, fst is the forcing state: the OU updates due at the step's start time are
 * applied first, and that driving field acts during every stage of the step. */
int or_step_forced(const or_cfg *c, double *w, double *S_prev, double *wig, double *scal, double *fst, double dt,
                   double *dt_used)
{
    if (check_cfg(c)) return OR_EINVAL;
    if (c->forcing_on && !fst) return OR_EINVAL;
    or_geo g;
    geo_init(&g, c);
    int s = c->rk_stages > 0 ? c->rk_stages : or_rk_stages(c->n);
    double al[36], be[36];
    if (or_rk_table(s, al, be)) return OR_EINVAL;
    size_t nw = (size_t)g.FT * g.ncell * g.M;
    int status = OR_OK;
    /* the limiter also acts on the state entering the step: after the first
     * step that state is a limited stage output, so this only changes
     * initial data (a projected discontinuity can be negative at points) */
    if (c->positivity_on) status |= or_positivity(c, w);
    if (c->av_on) status |= or_wiggle(c, w, S_prev, wig, scal[0], (long)scal[1]);
    if (c->forcing_on) status |= or_forcing_update(c, fst, scal[2]);
    if (!(dt > 0.0)) status |= or_max_dt(c, w, &dt);
    if (status & OR_EINVAL) return status;
    double *U[6], *L[6];
    for (int i = 0; i <= s; ++i) {
        U[i] = malloc(sizeof(double) * nw);
        L[i] = malloc(sizeof(double) * nw);
    }
    memcpy(U[0], w, sizeof(double) * nw);
    for (int i = 1; i <= s; ++i) {
        status |= or_rhs_forced(c, U[i - 1], c->av_on ? wig : NULL, c->forcing_on ? fst : NULL, L[i - 1]);
        for (size_t q = 0; q < nw; ++q) {
            double acc = 0.0;
            for (int k = 0; k < i; ++k) {
                if (al[i * 6 + k] != 0.0) acc += al[i * 6 + k] * U[k][q];
                if (be[i * 6 + k] != 0.0) acc += be[i * 6 + k] * dt * L[k][q];
            }
            U[i][q] = acc;
        }
        if (c->positivity_on) status |= or_positivity(c, U[i]);
    }
    memcpy(w, U[s], sizeof(double) * nw);
    for (int i = 0; i <= s; ++i) {
        free(U[i]);
        free(L[i]);
    }
    scal[0] = dt;
    scal[1] += 1.0;
    scal[2] += dt;
    if (dt_used) *dt_used = dt;
    return status;
}

int or_step(const or_cfg *c, double *w, double *S_prev, double *wig, double *scal, double dt, double *dt_used)
{
    return or_step_forced(c, w, S_prev, wig, scal, NULL, dt, dt_used);
}

/* basis values phi_l at arbitrary reference points xi[npts][d] -> out[npts][M] */
/* basis values phi_l at reference points xi[npts][d] -> out[npts][M] for either basis */
int or_basis_eval_b(int d, int n, int basis, int npts, const double *xi, double *out)
{
    int exps[OR_MAXM][3], mode_of[OR_MAXM];
    if (d < 2 || d > 3 || n < 0 || n > OR_MAXN) return OR_EINVAL;
    int M = mode_list(d, n, basis, exps, mode_of);
    for (int i = 0; i < npts; ++i)
        for (int l = 0; l < M; ++l) {
            double v = 1.0;
            for (int a = 0; a < d; ++a) v *= or_pt(exps[l][a], xi[i * d + a]);
            out[i * M + l] = v;
        }
    return OR_OK;
}

int or_basis_eval(int d, int n, int npts, const double *xi, double *out)
{
    int Q = n + 1, M = 1;
    for (int a = 0; a < d; ++a) M *= Q;
    for (int i = 0; i < npts; ++i)
        for (int l = 0; l < M; ++l) {
            int ll[3];
            unflat(l, Q, d, ll);
            double v = 1.0;
            for (int a = 0; a < d; ++a) v *= or_pt(ll[a], xi[i * d + a]);
            out[i * M + l] = v;
        }
    return OR_OK;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* recovered state ut[k][f] and physical gradient gt[k][3][f] at the points of
 * the face normal to `ax` between cells KL (left) and KR (right), exactly as
 * the right-hand side uses them (exposed for the recovery pins) */
int or_face_recovery(const or_cfg *c, const double *w, long KL, long KR, int ax, double *ut, double *gt)
{
    if (check_cfg(c)) return OR_EINVAL;
    or_geo g;
    geo_init(&g, c);
    or_tab T;
    if (tab_init(&T, g.d, g.n, g.M, (const int(*)[3])g.exps)) return OR_EINVAL;
    memset(gt, 0, sizeof(double) * T.NQF * 3 * g.NF);
    face_recovery(&T, &g, w, KL, KR, ax, ut, gt);
    tab_free(&T);
    return OR_OK;
}
