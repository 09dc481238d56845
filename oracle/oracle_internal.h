/* Oracle internals shared between the oracle's own translation units.
 * Test infrastructure only (see oracle.h).                              */
#ifndef GKS_ORACLE_INTERNAL_H
#define GKS_ORACLE_INTERNAL_H

#include "oracle.h"

namespace orc {

constexpr int kMaxU = 7;      /* highest power of u needed: 6 */
constexpr int kMaxV = 6;
constexpr int kMaxSolve = 128;

struct Tables {
    double u[kMaxU + 1];
    double v[kMaxV + 1];
    double w[kMaxV + 1];
    double xi[3];
};
/* m[which][i][k] = <x psi_i psi_k>, x in {1,u,v,w,uu,uv,uw} */
struct GSet { double m[7][5][5]; };
enum { G1 = 0, GU = 1, GV = 2, GW = 3, GUU = 4, GUV = 5, GUW = 6 };

struct Prim { double rho, U, V, W, p, lam; };

void gauss_moments_1d(double C, double lam, int half, int nmax, double *m);
void moment_tables(double U, double V, double W, double lam, double Nint,
                   int half, Tables *t);
double monomial_moment(const Tables &t, int a, int b, int d, int k);
void g_matrix(const Tables &t, int which, double G[5][5]);
void all_g(const Tables &t, GSet *g);
int solve_dense(int n, const double *A, const double *b, double *x);
void matvec5(const double G[5][5], const double *a, double *y);
Prim primitive(const double *Wc, double gamma);
double internal_dof(double gamma);
int slope(const Prim &p, double Nint, const double *dW, double *a);

/* flux.cpp */
int flux_gp(const orc_params &P, const double *sl, const double *sr,
            double dt, double *out30);

/* recon.cpp */
/* variant 0: reading A (63-entry data vectors); 1: reading B (72) */
double geno_misfit(const double *q0, const double *d, const double *a, int v, int variant);
double geno_chi(double sigma);
void recon5_cell(const double *q0, const double *dvec, double hx, double hy,
                 double hz, int nonlinear, double *out480, double *chi5, int variant = 0);
void recon2_cell(const double *q7, double hx, double hy, double hz,
                 int nonlinear, double *out120, double *phi5);
/* Gauss points of a face in normalised cell coordinates: face f (0..5 =
 * x-,x+,y-,y+,z-,z+), point k (0..3)                                     */
void face_gauss_point(int f, int k, double x[3]);
/* Face frame permutation: axis of the face-frame direction j (0 normal,
 * 1 and 2 tangential) for a face of normal axis d.                       */
int frame_axis(int d, int j);

}  // namespace orc

#endif
