/*
 * exact_euler.c -- exact solution of the Riemann problem for the 1-D Euler
 * equations of an ideal gas (test infrastructure only).
 *
 * Method: the star-region pressure p* is the root of
 *     f(p) = f_L(p) + f_R(p) + (u_R - u_L) = 0,
 * with f_K the shock (Rankine-Hugoniot) branch for p > p_K and the
 * rarefaction (isentropic Riemann invariant) branch for p <= p_K; the root is
 * found by Newton iteration, then the self-similar solution is sampled at
 * xi = x/t.  This is the textbook construction of Toro, "Riemann Solvers and
 * Numerical Methods for Fluid Dynamics", ch. 4, written here from the
 * gas-dynamics relations.  It pins the oracle on the B = 0 limit of the MHD
 * system, where the paper's scheme must converge to this solution.
 */
#include <math.h>

static double f_k(double p, double rk, double pk, double g, double *df)
{
    double ck = sqrt(g * pk / rk);
    if (p > pk) {
        double A = 2.0 / ((g + 1.0) * rk);
        double B = (g - 1.0) / (g + 1.0) * pk;
        double q = sqrt(A / (p + B));
        *df = q * (1.0 - 0.5 * (p - pk) / (p + B));
        return (p - pk) * q;
    } else {
        double pr = p / pk;
        *df = pow(pr, -(g + 1.0) / (2.0 * g)) / (rk * ck);
        return 2.0 * ck / (g - 1.0) * (pow(pr, (g - 1.0) / (2.0 * g)) - 1.0);
    }
}

/* Star-region pressure and velocity.  Returns the number of Newton steps, or
 * -1 if the data generate vacuum. */
int or_euler_star(double rl, double ul, double pl, double rr, double ur, double pr,
                  double g, double *ps, double *us)
{
    double cl = sqrt(g * pl / rl), cr = sqrt(g * pr / rr);
    double p, fl, fr, dfl, dfr;
    int it;
    if (2.0 * (cl + cr) / (g - 1.0) <= ur - ul)
        return -1;
    /* two-rarefaction guess: positive and exact when both waves rarefy */
    {
        double z = (g - 1.0) / (2.0 * g);
        p = pow((cl + cr - 0.5 * (g - 1.0) * (ur - ul)) /
                    (cl / pow(pl, z) + cr / pow(pr, z)),
                1.0 / z);
    }
    for (it = 1; it <= 200; it++) {
        double pn;
        fl = f_k(p, rl, pl, g, &dfl);
        fr = f_k(p, rr, pr, g, &dfr);
        pn = p - (fl + fr + ur - ul) / (dfl + dfr);
        if (pn <= 0.0)
            pn = 0.5 * p;
        if (fabs(pn - p) <= 1.0e-15 * 0.5 * (pn + p)) {
            p = pn;
            break;
        }
        p = pn;
    }
    fl = f_k(p, rl, pl, g, &dfl);
    fr = f_k(p, rr, pr, g, &dfr);
    *ps = p;
    *us = 0.5 * (ul + ur) + 0.5 * (fr - fl);
    return it;
}

/* Sample the exact solution at xi = x/t: out = (rho, u, p). */
int or_euler_sample(double rl, double ul, double pl, double rr, double ur, double pr,
                    double g, double xi, double *out)
{
    double ps, us, cl = sqrt(g * pl / rl), cr = sqrt(g * pr / rr);
    double gm = (g - 1.0) / (g + 1.0);
    int it = or_euler_star(rl, ul, pl, rr, ur, pr, g, &ps, &us);
    if (it < 0)
        return -1;
    if (xi <= us) { /* left of the contact */
        if (ps > pl) { /* left shock */
            double sl = ul - cl * sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g));
            if (xi <= sl) {
                out[0] = rl; out[1] = ul; out[2] = pl;
            } else {
                out[0] = rl * (ps / pl + gm) / (gm * ps / pl + 1.0);
                out[1] = us;
                out[2] = ps;
            }
        } else { /* left rarefaction */
            double csl = cl * pow(ps / pl, (g - 1.0) / (2.0 * g));
            double head = ul - cl, tail = us - csl;
            if (xi <= head) {
                out[0] = rl; out[1] = ul; out[2] = pl;
            } else if (xi >= tail) {
                out[0] = rl * pow(ps / pl, 1.0 / g);
                out[1] = us;
                out[2] = ps;
            } else {
                double c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - xi));
                out[1] = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + xi);
                out[0] = rl * pow(c / cl, 2.0 / (g - 1.0));
                out[2] = pl * pow(c / cl, 2.0 * g / (g - 1.0));
            }
        }
    } else { /* right of the contact */
        if (ps > pr) { /* right shock */
            double sr = ur + cr * sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g));
            if (xi >= sr) {
                out[0] = rr; out[1] = ur; out[2] = pr;
            } else {
                out[0] = rr * (ps / pr + gm) / (gm * ps / pr + 1.0);
                out[1] = us;
                out[2] = ps;
            }
        } else { /* right rarefaction */
            double csr = cr * pow(ps / pr, (g - 1.0) / (2.0 * g));
            double head = ur + cr, tail = us + csr;
            if (xi >= head) {
                out[0] = rr; out[1] = ur; out[2] = pr;
            } else if (xi <= tail) {
                out[0] = rr * pow(ps / pr, 1.0 / g);
                out[1] = us;
                out[2] = ps;
            } else {
                double c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - xi));
                out[1] = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + xi);
                out[0] = rr * pow(c / cr, 2.0 / (g - 1.0));
                out[2] = pr * pow(c / cr, 2.0 * g / (g - 1.0));
            }
        }
    }
    return it;
}
