// flopcount.cpp -- count the floating-point operations of the CPU oracle's
// building blocks (test infrastructure; run by oracle/flopcount.py).
//
// The oracle source is compiled as C++ with `double` replaced by a counting
// number type: every +, -, *, / and sqrt on it increments a counter, except
// a +, - or * with an exact-zero operand (fabs, fmin, fmax, copysign and
// comparisons are not counted as flops; exp is counted on its own).  The driver reads states (local 1-D order) from
// stdin and prints the average counts per call of or_mhd_riemann,
// or_mhd_char_predict (linear and PPM), or_mhd_prim2cons and
// or_mhd_cons2prim, then the average counts per face of the parabolic
// fluxes (Section 3.1): each conduction variant, viscosity and resistivity
// on their own, over the faces of a 4^3 patch of generic fields.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

namespace fc {
struct Counts {
    unsigned long long add = 0, mul = 0, div = 0, sqrt = 0, exp = 0;
};
static Counts g;

struct Flop {
    double v;
    Flop() = default;
    Flop(double x) : v(x) {}
};
// an operation with an exact-zero operand (the oracle's dense eigenvector
// matrices hold structural zeros) is not counted
inline Flop operator+(Flop a, Flop b) { if (a.v != 0.0 && b.v != 0.0) ++g.add; return Flop(a.v + b.v); }
inline Flop operator-(Flop a, Flop b) { if (a.v != 0.0 && b.v != 0.0) ++g.add; return Flop(a.v - b.v); }
inline Flop operator*(Flop a, Flop b) { if (a.v != 0.0 && b.v != 0.0) ++g.mul; return Flop(a.v * b.v); }
inline Flop operator/(Flop a, Flop b) { ++g.div; return Flop(a.v / b.v); }
inline Flop operator-(Flop a) { return Flop(-a.v); }
inline Flop &operator+=(Flop &a, Flop b) { a = a + b; return a; }
inline Flop &operator-=(Flop &a, Flop b) { a = a - b; return a; }
inline Flop &operator*=(Flop &a, Flop b) { a = a * b; return a; }
inline Flop &operator/=(Flop &a, Flop b) { a = a / b; return a; }
inline bool operator<(Flop a, Flop b) { return a.v < b.v; }
inline bool operator>(Flop a, Flop b) { return a.v > b.v; }
inline bool operator<=(Flop a, Flop b) { return a.v <= b.v; }
inline bool operator>=(Flop a, Flop b) { return a.v >= b.v; }
inline bool operator==(Flop a, Flop b) { return a.v == b.v; }
inline bool operator!=(Flop a, Flop b) { return a.v != b.v; }
inline Flop sqrt(Flop a) { ++g.sqrt; return Flop(std::sqrt(a.v)); }
inline Flop fabs(Flop a) { return Flop(std::fabs(a.v)); }
inline Flop fmin(Flop a, Flop b) { return Flop(std::fmin(a.v, b.v)); }
inline Flop fmax(Flop a, Flop b) { return Flop(std::fmax(a.v, b.v)); }
inline Flop copysign(Flop a, Flop b) { return Flop(std::copysign(a.v, b.v)); }
inline Flop exp(Flop a) { ++g.exp; return Flop(std::exp(a.v)); }
} // namespace fc

using fc::Flop;
using fc::sqrt;
using fc::fabs;
using fc::fmin;
using fc::fmax;
using fc::copysign;
using fc::exp;

#define double Flop
#include "ctu_oracle.c"
#include "srmhd_oracle.c"
#undef double

static double total(const fc::Counts &c)
{
    return (double)(c.add + c.mul + c.div + c.sqrt);
}

// Average flops of one parabolic face flux over the 3 x 64 faces of a 4^3
// patch (3-D) whose fields (rho, v, T, B) are drawn from a fixed xorshift64
// sequence: rho, T in [0.5, 1.5), v, B in [-1, 1).
static double face_count(double kappa, double kpar, double phi, double nu, double eta)
{
    grid_t G;
    grid_init(&G, 4, 4, 4, 3);
    const long nc = G.ncell;
    Flop *W = new Flop[8 * nc];
    unsigned long long s = 88172645463325252ull;
    auto rnd = [&]() {
        s ^= s << 13;
        s ^= s >> 7;
        s ^= s << 17;
        return (double)(s >> 11) * (1.0 / 9007199254740992.0);
    };
    for (long i = 0; i < nc; ++i) {
        W[i] = Flop(0.5 + rnd());
        for (int q = 1; q <= 3; ++q) W[q * nc + i] = Flop(2.0 * rnd() - 1.0);
        W[4 * nc + i] = Flop(0.5 + rnd());
        for (int q = 5; q <= 7; ++q) W[q * nc + i] = Flop(2.0 * rnd() - 1.0);
    }
    Flop h[3] = {Flop(0.25), Flop(0.25), Flop(0.25)};
    double tot = 0.0;
    int nf = 0;
    for (int k = 0; k < 4; ++k)
        for (int j = 0; j < 4; ++j)
            for (int i = 0; i < 4; ++i)
                for (int d = 0; d < 3; ++d) {
                    const int c[3] = {i, j, k};
                    Flop Pi[NVAR];
                    fc::g = fc::Counts();
                    parabolic_face(&G, W, h, Flop(kappa), Flop(kpar), Flop(phi), Flop(nu), Flop(eta), cidx(&G, c), d,
                                   Pi);
                    tot += total(fc::g);
                    ++nf;
                }
    delete[] W;
    return tot / nf;
}

// Relativistic MHD (srmhd_oracle.c): input K, Gamma, ch, dtdx, then K
// records of 3 x 9 primitive values (cells i - 1, i, i + 1, local order)
// and 9 conserved values of cell i.  Prints the average counts per call.
static int count_srmhd()
{
    int K;
    double gam, ch, dtdx;
    if (scanf("%d %lf %lf %lf", &K, &gam, &ch, &dtdx) != 4) return 1;
    double r_riem = 0, r_pred = 0, r_p2c = 0, r_c2p = 0, r_fs = 0;
    for (int k = 0; k < K; ++k) {
        double in[36];
        for (int i = 0; i < 36; ++i)
            if (scanf("%lf", &in[i]) != 1) return 1;
        Flop vs[27], U0[9], VL[9], VR[9], F[9], Vp[9], Vm[9], U[9], V[9], lm, lp;
        for (int i = 0; i < 27; ++i) vs[i] = Flop(in[i]);
        for (int q = 0; q < 9; ++q) {
            U0[q] = Flop(in[27 + q]);
            VL[q] = vs[9 + q];
            VR[q] = vs[18 + q];
        }
        fc::g = fc::Counts();
        or_srmhd_riemann(VL, VR, Flop(gam), Flop(ch), F);
        r_riem += total(fc::g);
        fc::g = fc::Counts();
        or_srmhd_mh_predict(vs, U0, Flop(gam), Flop(ch), Flop(dtdx), Vp, Vm);
        r_pred += total(fc::g);
        fc::g = fc::Counts();
        or_srmhd_prim2cons(VL, Flop(gam), U);
        r_p2c += total(fc::g);
        fc::g = fc::Counts();
        or_srmhd_cons2prim(U0, Flop(gam), V);
        r_c2p += total(fc::g);
        fc::g = fc::Counts();
        or_srmhd_fast_speeds(VL, Flop(gam), &lm, &lp);
        r_fs += total(fc::g);
    }
    printf("sr_riemann %.2f\nsr_predict %.2f\nsr_prim2cons %.2f\nsr_cons2prim %.2f\nsr_fast_speeds %.2f\n",
           r_riem / K, r_pred / K, r_p2c / K, r_c2p / K, r_fs / K);
    return 0;
}

int main(int argc, char **argv)
{
    if (argc > 1 && !strcmp(argv[1], "srmhd")) return count_srmhd();
    // input: count K, gamma, ch, dtdx, then K stencils of 5 x 9 values (local order)
    int K;
    double gam, ch, dtdx;
    if (scanf("%d %lf %lf %lf", &K, &gam, &ch, &dtdx) != 4) return 1;
    double *S = (double *)malloc(sizeof(double) * 45 * K);
    for (int i = 0; i < 45 * K; ++i)
        if (scanf("%lf", &S[i]) != 1) return 1;
    double r_riem = 0, r_pred0 = 0, r_pred1 = 0, r_p2c = 0, r_c2p = 0, r_cf = 0;
    double r_predv[4] = {0, 0, 0, 0};
    for (int k = 0; k < K; ++k) {
        Flop vs[45], VL[9], VR[9], F[9], Vp[9], Vm[9], U[9], V[9];
        for (int i = 0; i < 45; ++i) vs[i] = Flop(S[45 * k + i]);
        for (int q = 0; q < 9; ++q) {
            VL[q] = vs[18 + q];
            VR[q] = vs[27 + q];
        }
        fc::g = fc::Counts();
        or_mhd_riemann(VL, VR, Flop(gam), Flop(ch), F);
        r_riem += total(fc::g);
        fc::g = fc::Counts();
        or_mhd_char_predict(vs, Flop(gam), Flop(ch), Flop(dtdx), 0, 0, Vp, Vm);
        r_pred0 += total(fc::g);
        fc::g = fc::Counts();
        or_mhd_char_predict(vs, Flop(gam), Flop(ch), Flop(dtdx), 1, 0, Vp, Vm);
        r_pred1 += total(fc::g);
        for (int r = 2; r <= 5; ++r) {
            fc::g = fc::Counts();
            or_mhd_char_predict_dx(vs, Flop(gam), Flop(ch), Flop(dtdx), Flop(0.1), r, 0, Vp, Vm);
            r_predv[r - 2] += total(fc::g);
        }
        fc::g = fc::Counts();
        or_mhd_prim2cons(VL, Flop(gam), U);
        r_p2c += total(fc::g);
        fc::g = fc::Counts();
        or_mhd_cons2prim(U, Flop(gam), V);
        r_c2p += total(fc::g);
        fc::g = fc::Counts();
        or_mhd_cfast(VL, Flop(gam));
        r_cf += total(fc::g);
    }
    printf("riemann %.2f\npredict_linear %.2f\npredict_ppm %.2f\nprim2cons %.2f\ncons2prim %.2f\ncfast %.2f\n",
           r_riem / K, r_pred0 / K, r_pred1 / K, r_p2c / K, r_c2p / K, r_cf / K);
    printf("predict_minmod %.2f\npredict_harmonic %.2f\npredict_vanalbada %.2f\npredict_weno3 %.2f\n",
           r_predv[0] / K, r_predv[1] / K, r_predv[2] / K, r_predv[3] / K);
    printf("par_face_cond %.2f\npar_face_aniso %.2f\npar_face_sat %.2f\npar_face_sat_aniso %.2f\n",
           face_count(1e-3, 1e-3, 0.0, 0.0, 0.0), face_count(1e-3, 1e-2, 0.0, 0.0, 0.0),
           face_count(1e-3, 1e-3, 1e-2, 0.0, 0.0), face_count(1e-3, 1e-2, 1e-2, 0.0, 0.0));
    printf("par_face_visc %.2f\npar_face_res %.2f\n", face_count(0.0, 0.0, 0.0, 1e-3, 0.0),
           face_count(0.0, 0.0, 0.0, 0.0, 1e-3));
    // every combination of the terms, counted together (work the terms share,
    // the face means and differences, is counted once): par_mask_<c>_<v>_<r>
    // with c = none, cond, aniso, sat, sat_aniso and v, r = 0/1
    const char *cn[5] = {"none", "cond", "aniso", "sat", "sat_aniso"};
    const double ck[5][3] = {{0, 0, 0}, {1e-3, 1e-3, 0}, {1e-3, 1e-2, 0}, {1e-3, 1e-3, 1e-2}, {1e-3, 1e-2, 1e-2}};
    for (int c = 0; c < 5; ++c)
        for (int v = 0; v < 2; ++v)
            for (int r = 0; r < 2; ++r) {
                if (c == 0 && v == 0 && r == 0) continue;
                printf("par_mask_%s_%d_%d %.2f\n", cn[c], v, r,
                       face_count(ck[c][0], ck[c][1], ck[c][2], v ? 1e-3 : 0.0, r ? 1e-3 : 0.0));
            }
    return 0;
}
