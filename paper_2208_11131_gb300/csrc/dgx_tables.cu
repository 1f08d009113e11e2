// Host generation of the per-degree operator tables used by the kernels
// (see Tables<> in dgx_internal.h).  Computed in long double, then rounded
// once to FP64 and to FP32.
//
//  - Gauss-Legendre rule with n+1 points (Sec. 2.4): Newton iteration on
//    P_{n+1} from the asymptotic initial guess cos(pi (4i+3)/(4Q+2)).
//  - scaled Legendre basis Pt_l = sqrt(2l+1) P_l (Sec. 2.3 normalisation).
//  - Because the Q-point rule integrates Pt_a Pt_b exactly, the inverse of
//    the collocation matrix B[i][a] = Pt_a(x_i) is Binv[a][i] = g_i B[i][a] / 2;
//    every modal functional c_a turns into the nodal functional sum_a c_a Binv[a][i].
//  - interface recovery (Sec. 3.2, Eq. basisprojection, read with prefactor
//    1/2 in the K* unit coordinate and A+ argument 2 f x - 1): the joint
//    coefficient q_l = 1/2 sum_a (A-_{a,l} w-_a + A+_{a,l} w+_a), l = 0..n+1,
//    evaluated at the interface (K* coordinate 0): value sum_l q_l Pt_l(0),
//    normal derivative sum_l q_l Pt_l'(0) / (f h).  f = 3/4 for n <= 2, else 1.
#include <math.h>

#include "dgx_internal.h"

namespace dgx {

namespace {

typedef long double LD;

LD legendre(int l, LD x, LD *dp)
{
    // three-term recurrence for P_l and its derivative
    LD p0 = 1.0L, p1 = x, d0 = 0.0L, d1 = 1.0L;
    if (l == 0) {
        if (dp) *dp = 0.0L;
        return 1.0L;
    }
    for (int k = 2; k <= l; ++k) {
        LD p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        LD d2 = d0 + (2 * k - 1) * p1;
        p0 = p1;
        p1 = p2;
        d0 = d1;
        d1 = d2;
    }
    if (dp) *dp = d1;
    return p1;
}

LD pt(int l, LD x) { return sqrtl(2.0L * l + 1.0L) * legendre(l, x, nullptr); }
LD dpt(int l, LD x)
{
    LD d;
    legendre(l, x, &d);
    return sqrtl(2.0L * l + 1.0L) * d;
}

void gauss_rule(int q, LD *x, LD *w)
{
    const LD pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < q; ++i) {
        LD z = cosl(pi * (4 * i + 3) / (4 * q + 2));
        for (int it = 0; it < 60; ++it) {
            LD d;
            LD p = legendre(q, z, &d);
            LD step = p / d;
            z -= step;
            if (fabsl(step) <= 1e-24L) break;
        }
        LD d;
        legendre(q, z, &d);
        x[q - 1 - i] = z;  // ascending
        w[q - 1 - i] = 2.0L / ((1.0L - z * z) * d * d);
    }
}

}  // namespace

void make_tables(int n, Tables<double> *td, Tables<float> *tf)
{
    const int Q = n + 1;
    LD x[kMaxQ], g[kMaxQ];
    gauss_rule(Q, x, g);
    LD B[kMaxQ][kMaxQ], Binv[kMaxQ][kMaxQ], Dm[kMaxQ][kMaxQ], Dn[kMaxQ][kMaxQ];
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < Q; ++a) {
            B[i][a] = pt(a, x[i]);
            Dm[i][a] = dpt(a, x[i]);
        }
    for (int a = 0; a < Q; ++a)
        for (int i = 0; i < Q; ++i) Binv[a][i] = 0.5L * g[i] * B[i][a];
    for (int i = 0; i < Q; ++i)
        for (int m = 0; m < Q; ++m) {
            LD s = 0.0L;
            for (int a = 0; a < Q; ++a) s += Dm[i][a] * Binv[a][m];
            Dn[i][m] = s;
        }
    // nodal functional from a modal one
    auto nodal = [&](const LD *c, LD *out) {
        for (int m = 0; m < Q; ++m) {
            LD s = 0.0L;
            for (int a = 0; a < Q; ++a) s += c[a] * Binv[a][m];
            out[m] = s;
        }
    };
    LD tp[kMaxQ], tm[kMaxQ], Lp[kMaxQ], Lm[kMaxQ];
    for (int a = 0; a < Q; ++a) {
        tp[a] = pt(a, 1.0L);
        tm[a] = pt(a, -1.0L);
    }
    nodal(tp, Lp);
    nodal(tm, Lm);

    // recovery overlap integrals with a 12-point rule on each half interval
    const LD f = n <= 2 ? 0.75L : 1.0L;
    LD xr[12], wr[12];
    gauss_rule(12, xr, wr);
    LD cm[kMaxQ], cp[kMaxQ], dm[kMaxQ], dp[kMaxQ];
    for (int a = 0; a < Q; ++a) {
        cm[a] = cp[a] = dm[a] = dp[a] = 0.0L;
        for (int l = 0; l <= n + 1; ++l) {
            LD Aml = 0.0L, Apl = 0.0L;
            for (int j = 0; j < 12; ++j) {
                LD sl = -0.5L + 0.5L * xr[j];  // in [-1, 0]
                LD sr = 0.5L + 0.5L * xr[j];   // in [0, 1]
                Aml += 0.5L * wr[j] * pt(a, 2.0L * f * sl + 1.0L) * pt(l, sl);
                Apl += 0.5L * wr[j] * pt(a, 2.0L * f * sr - 1.0L) * pt(l, sr);
            }
            cm[a] += 0.5L * Aml * pt(l, 0.0L);
            cp[a] += 0.5L * Apl * pt(l, 0.0L);
            dm[a] += 0.5L * Aml * dpt(l, 0.0L);
            dp[a] += 0.5L * Apl * dpt(l, 0.0L);
        }
    }
    LD Cm[kMaxQ], Cp[kMaxQ], DMn[kMaxQ], DPn[kMaxQ];
    nodal(cm, Cm);
    nodal(cp, Cp);
    nodal(dm, DMn);
    nodal(dp, DPn);

    Tables<double> T{};
    for (int i = 0; i < Q; ++i) {
        T.G[i] = (double)g[i];
        T.Lp[i] = (double)Lp[i];
        T.Lm[i] = (double)Lm[i];
        T.Cm[i] = (double)Cm[i];
        T.Cp[i] = (double)Cp[i];
        T.Dm[i] = (double)DMn[i];
        T.Dp[i] = (double)DPn[i];
        for (int m = 0; m < Q; ++m) {
            T.B[i][m] = (double)B[i][m];
            T.Dn[i][m] = (double)Dn[i][m];
            T.Wd[i][m] = (double)(g[m] * Dn[m][i]);
        }
    }
    T.inv_f = (double)(1.0L / f);
    *td = T;
    Tables<float> F{};
    for (int i = 0; i < Q; ++i) {
        F.G[i] = (float)g[i];
        F.Lp[i] = (float)Lp[i];
        F.Lm[i] = (float)Lm[i];
        F.Cm[i] = (float)Cm[i];
        F.Cp[i] = (float)Cp[i];
        F.Dm[i] = (float)DMn[i];
        F.Dp[i] = (float)DPn[i];
        for (int m = 0; m < Q; ++m) {
            F.B[i][m] = (float)B[i][m];
            F.Dn[i][m] = (float)Dn[i][m];
            F.Wd[i][m] = (float)(g[m] * Dn[m][i]);
        }
    }
    F.inv_f = (float)(1.0L / f);
    *tf = F;
}

void gauss_nodes(int q, double *x)
{
    LD xl[kMaxQ + 2], wl[kMaxQ + 2];
    gauss_rule(q, xl, wl);
    for (int i = 0; i < q; ++i) x[i] = (double)xl[i];
}

}  // namespace dgx
