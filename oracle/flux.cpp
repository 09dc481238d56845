/*
 * Oracle: gas-kinetic interface flux at one Gauss point (Sec. 2).
 * Test infrastructure only (see oracle.h).
 *
 * Follows the paper's order:
 *   Eq. flux          time-accurate f(x_G, t) from g0, g_l, g_r and slopes;
 *   (after Eq. flux)  f^n, f_t^n from the time integrals fbar(dt), fbar(dt/2);
 *   Eq. deri-t-f      F^n, F_t^n as moments of f^n, f_t^n;
 *   Sec. 3.4          interface values Q^l, Q^r from the blend of the
 *                     equilibrium and one-sided evolutions;
 *   Sec. 4            collision time tau.
 * Everything is in the face frame: u is the particle velocity along the
 * face normal, (v, w) along the two tangential axes.
 */
#include "oracle_internal.h"

#include <cmath>
#include <cstring>

namespace orc {
namespace {

/* Time integrals over [0, T] of the six coefficient functions of Eq. flux:
 *   c1: 1 - e^{-t/tau}              (g0)
 *   c2: (t + tau) e^{-t/tau} - tau   (abar.u g0)
 *   c3: t - tau + tau e^{-t/tau}     (Abar g0)
 *   c4: e^{-t/tau}                   (g_l H + g_r (1-H))
 *   c5: -(tau + t) e^{-t/tau}        (a^{l,r}.u g_{l,r})
 *   c6: -tau e^{-t/tau}              (A^{l,r} g_{l,r})
 * With x = T/tau and E = 1 - e^{-x}:
 *   c1 = T - tau E, c2 = 2 tau^2 E - tau T (2 - E), c3 = T^2/2 - tau T + tau^2 E,
 *   c4 = tau E, c5 = -2 tau^2 E + tau T (1 - E), c6 = -tau^2 E.
 * c1..c3 cancel for small x; there their Taylor series are summed.      */
void time_coeffs(double T, double tau, double c[6]) {
    if (tau == 0.0) {  /* tau -> 0 limit */
        c[0] = T; c[1] = 0.0; c[2] = 0.5 * T * T;
        c[3] = 0.0; c[4] = 0.0; c[5] = 0.0;
        return;
    }
    const double x = T / tau;
    const double E = -std::expm1(-x);
    const double t2 = tau * tau;
    if (x < 1.0) {
        /* c1/tau = sum_{n>=2} (-1)^n x^n/n!
         * c2/tau^2 = sum_{n>=3} (-1)^n (n-2) x^n/n!
         * c3/tau^2 = sum_{n>=3} (-1)^{n+1} x^n/n!                           */
        double s1 = 0.0, s2 = 0.0, s3 = 0.0;
        double term = x;  /* x^n/n! at n = 1 */
        for (int n = 2; n <= 30; ++n) {
            term *= x / n;
            const double sg = (n % 2 == 0) ? 1.0 : -1.0;
            s1 += sg * term;
            if (n >= 3) {
                s2 += sg * (n - 2) * term;
                s3 -= sg * term;
            }
        }
        c[0] = tau * s1;
        c[1] = t2 * s2;
        c[2] = t2 * s3;
    } else {
        c[0] = T - tau * E;
        c[1] = 2.0 * t2 * E - tau * T * (2.0 - E);
        c[2] = 0.5 * T * T - tau * T + t2 * E;
    }
    c[3] = tau * E;
    c[4] = -2.0 * t2 * E + tau * T * (1.0 - E);
    c[5] = -t2 * E;
}

double viscosity(const orc_params &P, double rho, double p) {
    if (P.mu_law == 0) return P.mu0;
    /* Sutherland law of Sec. 4.2, temperature normalised by T_ref */
    const double th = (p / rho) / P.T_ref;
    return P.mu0 * 1.4042 * th * std::sqrt(th) / (th + 0.4042);
}

struct FluxWork {
    Prim l, r, z;            /* left, right, interface equilibrium */
    double al[3][5], ar[3][5], abar[3][5];
    double Al[5], Ar[5], Abar[5];
    double W0[5], dW0[3][5];
    double dtWl[5], dtWr[5], dtW0[5];
    double X[6][5];          /* flux moments of the six terms of Eq. flux   */
    double Y[6][5];          /* conserved moments of the same terms          */
    double tau;
};

void add_scaled(double *y, double s, const double *x) {
    for (int i = 0; i < 5; ++i) y[i] += s * x[i];
}

/* Everything except the time integration: slopes, equilibrium state,
 * collision time and the moment vectors of each term of Eq. flux.       */
int prepare(const orc_params &P, const double *sl, const double *sr, double dt,
            FluxWork *w) {
    const double Nint = internal_dof(P.gamma);
    w->l = primitive(sl, P.gamma);
    w->r = primitive(sr, P.gamma);
    if (!(w->l.rho > 0 && w->l.p > 0 && w->r.rho > 0 && w->r.p > 0)) return -3;

    /* one-sided Maxwellian slopes a^{l,r}_j: <(a.psi) psi> = dW/rho       */
    for (int j = 0; j < 3; ++j) {
        if (slope(w->l, Nint, sl + 5 * (j + 1), w->al[j])) return -3;
        if (slope(w->r, Nint, sr + 5 * (j + 1), w->ar[j])) return -3;
    }
    /* full-space moments of g_l, g_r; A^{l,r} from the compatibility
     * condition int (a.u + A) psi g = 0                                   */
    Tables tl, tr, thl, thr;
    moment_tables(w->l.U, w->l.V, w->l.W, w->l.lam, Nint, 0, &tl);
    moment_tables(w->r.U, w->r.V, w->r.W, w->r.lam, Nint, 0, &tr);
    static thread_local GSet gl, gr, hl, hr, g0;
    all_g(tl, &gl);
    all_g(tr, &gr);
    {
        double Tl[5], Tr[5], tmp[5];
        for (int i = 0; i < 5; ++i) Tl[i] = Tr[i] = 0.0;
        for (int j = 0; j < 3; ++j) {
            matvec5(gl.m[GU + j], w->al[j], tmp); add_scaled(Tl, 1.0, tmp);
            matvec5(gr.m[GU + j], w->ar[j], tmp); add_scaled(Tr, 1.0, tmp);
        }
        double ml[5], mr[5];
        for (int i = 0; i < 5; ++i) { ml[i] = -Tl[i]; mr[i] = -Tr[i]; }
        if (solve_dense(5, &gl.m[G1][0][0], ml, w->Al)) return -3;
        if (solve_dense(5, &gr.m[G1][0][0], mr, w->Ar)) return -3;
        /* Euler time derivatives of the one-sided states: int A g psi */
        double t5[5];
        matvec5(gl.m[G1], w->Al, t5);
        for (int i = 0; i < 5; ++i) w->dtWl[i] = w->l.rho * t5[i];
        matvec5(gr.m[G1], w->Ar, t5);
        for (int i = 0; i < 5; ++i) w->dtWr[i] = w->r.rho * t5[i];
    }
    /* half-space moments: g_l over u > 0, g_r over u < 0                   */
    moment_tables(w->l.U, w->l.V, w->l.W, w->l.lam, Nint, +1, &thl);
    moment_tables(w->r.U, w->r.V, w->r.W, w->r.lam, Nint, -1, &thr);
    all_g(thl, &hl);
    all_g(thr, &hr);

    /* interface equilibrium: W0 = int_{u>0} psi g_l + int_{u<0} psi g_r   */
    for (int i = 0; i < 5; ++i)
        w->W0[i] = w->l.rho * hl.m[G1][i][0] + w->r.rho * hr.m[G1][i][0];
    /* its spatial derivatives by the same collision of the slopes (R6)    */
    for (int j = 0; j < 3; ++j) {
        double tl5[5], tr5[5];
        matvec5(hl.m[G1], w->al[j], tl5);
        matvec5(hr.m[G1], w->ar[j], tr5);
        for (int i = 0; i < 5; ++i)
            w->dW0[j][i] = w->l.rho * tl5[i] + w->r.rho * tr5[i];
    }
    w->z = primitive(w->W0, P.gamma);
    if (!(w->z.rho > 0 && w->z.p > 0)) return -3;
    for (int j = 0; j < 3; ++j)
        if (slope(w->z, Nint, w->dW0[j], w->abar[j])) return -3;
    Tables t0;
    moment_tables(w->z.U, w->z.V, w->z.W, w->z.lam, Nint, 0, &t0);
    all_g(t0, &g0);
    double T0v[5] = {0, 0, 0, 0, 0}, tmp[5];
    for (int j = 0; j < 3; ++j) {
        matvec5(g0.m[GU + j], w->abar[j], tmp);
        add_scaled(T0v, 1.0, tmp);
    }
    {
        double m0[5];
        for (int i = 0; i < 5; ++i) m0[i] = -T0v[i];
        if (solve_dense(5, &g0.m[G1][0][0], m0, w->Abar)) return -3;
        double t5[5];
        matvec5(g0.m[G1], w->Abar, t5);
        for (int i = 0; i < 5; ++i) w->dtW0[i] = w->z.rho * t5[i];
    }

    /* collision time (Sec. 4)                                              */
    const double dpr = std::fabs((w->l.p - w->r.p) / (w->l.p + w->r.p));
    if (P.inviscid)
        w->tau = P.eps_tau * dt + P.C_tau * dpr * dt;
    else
        w->tau = viscosity(P, w->z.rho, w->z.p) / w->z.p + P.C_tau * dpr * dt;

    /* moment vectors of the six terms of Eq. flux: X with the extra u of
     * the flux (Eq. flux-macro), Y without it (Eq. Q-macro)               */
    const double rl = w->l.rho, rr = w->r.rho, r0 = w->z.rho;
    for (int k = 0; k < 6; ++k)
        for (int i = 0; i < 5; ++i) w->X[k][i] = w->Y[k][i] = 0.0;
    /* term 1: g0 */
    for (int i = 0; i < 5; ++i) {
        w->X[0][i] = r0 * g0.m[GU][i][0];
        w->Y[0][i] = r0 * g0.m[G1][i][0];
    }
    /* term 2: (abar_1 u + abar_2 v + abar_3 w) g0 */
    for (int j = 0; j < 3; ++j) {
        matvec5(g0.m[GUU + j], w->abar[j], tmp); add_scaled(w->X[1], r0, tmp);
        matvec5(g0.m[GU + j], w->abar[j], tmp);  add_scaled(w->Y[1], r0, tmp);
    }
    /* term 3: Abar g0 */
    matvec5(g0.m[GU], w->Abar, tmp); add_scaled(w->X[2], r0, tmp);
    matvec5(g0.m[G1], w->Abar, tmp); add_scaled(w->Y[2], r0, tmp);
    /* term 4: g_l H(u) + g_r (1 - H(u)) */
    for (int i = 0; i < 5; ++i) {
        w->X[3][i] = rl * hl.m[GU][i][0] + rr * hr.m[GU][i][0];
        w->Y[3][i] = rl * hl.m[G1][i][0] + rr * hr.m[G1][i][0];
    }
    /* term 5: (a^s_1 u + a^s_2 v + a^s_3 w) g_s on its half space */
    for (int j = 0; j < 3; ++j) {
        matvec5(hl.m[GUU + j], w->al[j], tmp); add_scaled(w->X[4], rl, tmp);
        matvec5(hr.m[GUU + j], w->ar[j], tmp); add_scaled(w->X[4], rr, tmp);
        matvec5(hl.m[GU + j], w->al[j], tmp);  add_scaled(w->Y[4], rl, tmp);
        matvec5(hr.m[GU + j], w->ar[j], tmp);  add_scaled(w->Y[4], rr, tmp);
    }
    /* term 6: A^s g_s on its half space */
    matvec5(hl.m[GU], w->Al, tmp); add_scaled(w->X[5], rl, tmp);
    matvec5(hr.m[GU], w->Ar, tmp); add_scaled(w->X[5], rr, tmp);
    matvec5(hl.m[G1], w->Al, tmp); add_scaled(w->Y[5], rl, tmp);
    matvec5(hr.m[G1], w->Ar, tmp); add_scaled(w->Y[5], rr, tmp);
    return 0;
}

/* fbar(T): flux and conserved moments of f integrated over [0, T]; then
 * the Prandtl correction of the energy flux (reading R7).              */
void integrate(const orc_params &P, const FluxWork &w, double T, double *Fb,
               double *Wb, double *FbPr) {
    double c[6];
    time_coeffs(T, w.tau, c);
    for (int i = 0; i < 5; ++i) {
        double f = 0.0, q = 0.0;
        for (int k = 0; k < 6; ++k) {
            f += c[k] * w.X[k][i];
            q += c[k] * w.Y[k][i];
        }
        Fb[i] = f;
        Wb[i] = q;
    }
    /* heat flux q = 1/2 int (u - U0)((u-U0)^2 + (v-V0)^2 + (w-W0)^2 + xi^2) f
     * written through the flux and conserved moments of f                */
    const double U0 = w.z.U, V0 = w.z.V, W0 = w.z.W;
    const double q = (Fb[4] - U0 * Wb[4])
                   - (U0 * (Fb[1] - U0 * Wb[1]) + V0 * (Fb[2] - U0 * Wb[2]) +
                      W0 * (Fb[3] - U0 * Wb[3]))
                   + 0.5 * (U0 * U0 + V0 * V0 + W0 * W0) * (Fb[0] - U0 * Wb[0]);
    for (int i = 0; i < 5; ++i) FbPr[i] = Fb[i];
    FbPr[4] += (1.0 / P.Pr - 1.0) * q;
}

}  // namespace

int flux_gp(const orc_params &P, const double *sl, const double *sr, double dt,
            double *out) {
    static thread_local FluxWork w;
    const int rc = prepare(P, sl, sr, dt, &w);
    if (rc) return rc;
    double Fa[5], Wa[5], Pa[5], Fh[5], Wh[5], Ph[5];
    integrate(P, w, dt, Fa, Wa, Pa);
    integrate(P, w, 0.5 * dt, Fh, Wh, Ph);
    /* f^n = (4 fbar(dt/2) - fbar(dt))/dt, f_t^n = 4 (fbar(dt) - 2 fbar(dt/2))/dt^2 */
    for (int i = 0; i < 5; ++i) {
        out[i] = (4.0 * Ph[i] - Pa[i]) / dt;
        out[5 + i] = 4.0 * (Pa[i] - 2.0 * Ph[i]) / (dt * dt);
    }
    /* interface values (Sec. 3.4): Q^s(t) = (1-e) Q^e(t) + e Q_0^s(t)    */
    const double dpr = std::fabs((w.l.p - w.r.p) / (w.l.p + w.r.p));
    const double tau0 = P.C_tau * dpr * dt;
    const double e = (tau0 > 0.0) ? std::exp(-dt / tau0) : 0.0;
    for (int i = 0; i < 5; ++i) {
        out[10 + i] = (1.0 - e) * w.W0[i] + e * sl[i];
        out[15 + i] = (1.0 - e) * w.dtW0[i] + e * w.dtWl[i];
        out[20 + i] = (1.0 - e) * w.W0[i] + e * sr[i];
        out[25 + i] = (1.0 - e) * w.dtW0[i] + e * w.dtWr[i];
    }
    return 0;
}

}  // namespace orc

extern "C" int orc_flux_gp(const orc_params *P, const double *s_l,
                           const double *s_r, double dt, double *out30) {
    return orc::flux_gp(*P, s_l, s_r, dt, out30);
}

extern "C" int orc_fbar(const orc_params *P, const double *s_l,
                        const double *s_r, double dt, double T, double *out20) {
    static thread_local orc::FluxWork w;
    const int rc = orc::prepare(*P, s_l, s_r, dt, &w);
    if (rc) return rc;
    orc::integrate(*P, w, T, out20, out20 + 5, out20 + 10);
    out20[15] = w.tau;
    out20[16] = w.z.rho;
    out20[17] = w.z.U;
    out20[18] = w.z.V;
    out20[19] = w.z.W;
    return 0;
}
