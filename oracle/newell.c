/*
 * ORACLE (test infrastructure only): FP64 demagnetising tensor of a
 * rectangular cell, used by the CPU oracle of the micromagnetic hot path.
 * Only the tests, the smoke check and the timed CPU baseline may load it.
 *
 * What it computes (Methods, "Physics and discretization": open-boundary
 * demagnetisation by FFT convolution with the Newell tensor): the
 * cell-averaged field of a uniformly magnetised cell,
 *
 *   N_ab(R) = -1/(4 pi V) * Int_{V_target} Int_{V_source} K_ab(r - r') dr' dr,
 *   K_ab(r) = 3 r_a r_b / |r|^5 - delta_ab / |r|^3,      H_a = -sum_b N_ab M_b.
 *
 * Two evaluations of the same integral:
 *  - near field: the closed form of Newell, Williams & Dunlop (1993), a
 *    27-point second difference (weights 2,-1,-1 per axis) of the auxiliary
 *    functions f (diagonal) and g (off-diagonal);
 *  - far field: the double box integral collapses to one integral of K over
 *    the tent (box autocorrelation) T_d(t) = dx_d - |t| on |t| <= dx_d per
 *    axis; each tent half is integrated by n-point Gauss-Legendre, so the
 *    integrand is analytic on every sub-box.
 * The closed form loses about six digits to cancellation by 10 cells; the
 * quadrature converges geometrically with distance, so each regime is used
 * where it is accurate.  Displacements are in metres, cell sizes in metres.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Newell f: even in x, y, z (evaluated on |x|, |y|, |z|). */
double oracle_newell_f(double x, double y, double z)
{
    x = fabs(x); y = fabs(y); z = fabs(z);
    const double x2 = x * x, y2 = y * y, z2 = z * z;
    const double R = sqrt(x2 + y2 + z2);
    double f = (2.0 * x2 - y2 - z2) * R / 6.0;
    if (y > 0.0 && (x2 + z2) > 0.0)
        f += 0.5 * y * (z2 - x2) * asinh(y / sqrt(x2 + z2));
    if (z > 0.0 && (x2 + y2) > 0.0)
        f += 0.5 * z * (y2 - x2) * asinh(z / sqrt(x2 + y2));
    if (x > 0.0 && y > 0.0 && z > 0.0)
        f -= x * y * z * atan(y * z / (x * R));
    return f;
}

/* Newell g: odd in x and in y, even in z. */
double oracle_newell_g(double x, double y, double z)
{
    double s = 1.0;
    if (x < 0.0) { s = -s; x = -x; }
    if (y < 0.0) { s = -s; y = -y; }
    z = fabs(z);
    const double x2 = x * x, y2 = y * y, z2 = z * z;
    const double R = sqrt(x2 + y2 + z2);
    double g = -x * y * R / 3.0;
    if (z > 0.0 && (x2 + y2) > 0.0)
        g += x * y * z * asinh(z / sqrt(x2 + y2));
    if (x > 0.0 && (y2 + z2) > 0.0)
        g += y * (3.0 * z2 - y2) * asinh(x / sqrt(y2 + z2)) / 6.0;
    if (y > 0.0 && (x2 + z2) > 0.0)
        g += x * (3.0 * z2 - x2) * asinh(y / sqrt(x2 + z2)) / 6.0;
    if (z > 0.0 && x > 0.0 && y > 0.0)
        g -= z2 * z * atan(x * y / (z * R)) / 6.0;
    if (y > 0.0 && x > 0.0 && z > 0.0)
        g -= 0.5 * z * y2 * atan(x * z / (y * R));
    if (x > 0.0 && y > 0.0 && z > 0.0)
        g -= 0.5 * z * x2 * atan(y * z / (x * R));
    return s * g;
}

typedef double (*aux_fn)(double, double, double);

/* 27-point second difference of an auxiliary function. */
static double second_difference(aux_fn F, double X, double Y, double Z,
                                double hx, double hy, double hz)
{
    static const double w[3] = {-1.0, 2.0, -1.0};
    double acc = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                acc += w[i] * w[j] * w[k] *
                       F(X + (i - 1) * hx, Y + (j - 1) * hy, Z + (k - 1) * hz);
    return acc;
}

/*
 * Closed form at displacement (X,Y,Z), cell (dx,dy,dz).  out[6] =
 * xx, yy, zz, xy, xz, yz.  Lengths are rescaled by the largest cell edge
 * first (the tensor is scale invariant).
 */
void oracle_newell_analytic(double X, double Y, double Z,
                            double dx, double dy, double dz, double *out)
{
    const double s = fmax(dx, fmax(dy, dz));
    X /= s; Y /= s; Z /= s; dx /= s; dy /= s; dz /= s;
    const double c = 1.0 / (4.0 * M_PI * dx * dy * dz);
    /* N_xx uses f(x,y,z); N_yy = f with x<->y; N_zz = f with x<->z. */
    out[0] = c * second_difference(oracle_newell_f, X, Y, Z, dx, dy, dz);
    /* permuted: f(Y, X, Z) with steps (dy, dx, dz) */
    {
        static const double w[3] = {-1.0, 2.0, -1.0};
        double ayy = 0.0, azz = 0.0, axz = 0.0, ayz = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    const double ww = w[i] * w[j] * w[k];
                    const double x = X + (i - 1) * dx, y = Y + (j - 1) * dy, z = Z + (k - 1) * dz;
                    ayy += ww * oracle_newell_f(y, x, z);
                    azz += ww * oracle_newell_f(z, y, x);
                    axz += ww * oracle_newell_g(x, z, y);
                    ayz += ww * oracle_newell_g(y, z, x);
                }
        out[1] = c * ayy;
        out[2] = c * azz;
        out[4] = c * axz;
        out[5] = c * ayz;
    }
    out[3] = c * second_difference(oracle_newell_g, X, Y, Z, dx, dy, dz);
}

/* Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_n. */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double t = cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            /* p1 = P_n(t), p0 = P_{n-1}(t) */
            double dp = n * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        double p0 = 1.0, p1 = t;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = p2;
        }
        double dp = n * (t * p1 - p0) / (t * t - 1.0);
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

#define MAXQ 24

/*
 * Tent-weighted quadrature with nq Gauss points per tent half (2*nq per
 * axis).  Valid only when the tent support excludes the origin.
 */
void oracle_newell_quadrature(double X, double Y, double Z,
                              double dx, double dy, double dz, int nq, double *out)
{
    const double s = fmax(dx, fmax(dy, dz));
    X /= s; Y /= s; Z /= s; dx /= s; dy /= s; dz /= s;
    if (nq > MAXQ) nq = MAXQ;
    double gx[MAXQ], gw[MAXQ];
    gauss_legendre(nq, gx, gw);
    const double h[3] = {dx, dy, dz};
    double t[3][2 * MAXQ], wt[3][2 * MAXQ];
    for (int d = 0; d < 3; ++d)
        for (int q = 0; q < nq; ++q) {
            /* t = +-h(1+xi)/2, tent weight h(1-xi)/2, Jacobian h/2 */
            const double tt = 0.5 * h[d] * (1.0 + gx[q]);
            const double ww = gw[q] * 0.25 * h[d] * h[d] * (1.0 - gx[q]);
            t[d][2 * q] = tt;  wt[d][2 * q] = ww;
            t[d][2 * q + 1] = -tt; wt[d][2 * q + 1] = ww;
        }
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 2 * nq; ++i)
        for (int j = 0; j < 2 * nq; ++j)
            for (int k = 0; k < 2 * nq; ++k) {
                const double rx = X + t[0][i], ry = Y + t[1][j], rz = Z + t[2][k];
                const double r2 = rx * rx + ry * ry + rz * rz;
                const double ir2 = 1.0 / r2;
                const double ir3 = ir2 / sqrt(r2);
                const double ir5 = ir3 * ir2;
                const double w = wt[0][i] * wt[1][j] * wt[2][k];
                acc[0] += w * (3.0 * rx * rx * ir5 - ir3);
                acc[1] += w * (3.0 * ry * ry * ir5 - ir3);
                acc[2] += w * (3.0 * rz * rz * ir5 - ir3);
                acc[3] += w * (3.0 * rx * ry * ir5);
                acc[4] += w * (3.0 * rx * rz * ir5);
                acc[5] += w * (3.0 * ry * rz * ir5);
            }
    const double c = -1.0 / (4.0 * M_PI * dx * dy * dz);
    for (int a = 0; a < 6; ++a) out[a] = c * acc[a];
}

/*
 * The oracle's choice of evaluation at one displacement, by distance d in
 * units of the largest cell edge: closed form for d <= 2 (cancellation
 * costs ~1e-13 relative there for cells of aspect ratio <= 2, 1.5e-11 at
 * aspect ratio 6), quadrature beyond with 16 / 12 / 6 / 4 / 3 points per
 * tent half for d in (2,3], (3,8], (8,32], (32,128], > 128.  The
 * Gauss-Legendre error decays like rho^(-2n) with rho ~ 4d for these tents,
 * so every band is converged to ~5e-14 relative.
 */
void oracle_newell_at(double X, double Y, double Z,
                      double dx, double dy, double dz, double *out)
{
    const double s = fmax(dx, fmax(dy, dz));
    const double d = sqrt(X * X + Y * Y + Z * Z) / s;
    if (d <= 2.0) {
        oracle_newell_analytic(X, Y, Z, dx, dy, dz, out);
        return;
    }
    int nq = d <= 3.0 ? 16 : d <= 8.0 ? 12 : d <= 32.0 ? 6 : d <= 128.0 ? 4 : 3;
    oracle_newell_quadrature(X, Y, Z, dx, dy, dz, nq, out);
}

/*
 * Tensor on the non-negative octant of displacements i<nx, j<ny, k<nz:
 * out[a][k][j][i] (component-major, x fastest), a in xx,yy,zz,xy,xz,yz.
 * The other octants follow from parity (diagonal even in every axis;
 * xy odd in x and y, xz odd in x and z, yz odd in y and z).
 */
void oracle_newell_octant(int nx, int ny, int nz, double dx, double dy, double dz,
                          double *out)
{
    const long n = (long)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 64)
    for (long idx = 0; idx < n; ++idx) {
        const int i = (int)(idx % nx);
        const int j = (int)((idx / nx) % ny);
        const int k = (int)(idx / ((long)nx * ny));
        double v[6];
        oracle_newell_at(i * dx, j * dy, k * dz, dx, dy, dz, v);
        for (int a = 0; a < 6; ++a) out[a * n + idx] = v[a];
    }
}

/* Same, at an arbitrary list of integer displacements (i,j,k). */
void oracle_newell_list(long count, const int *ijk, double dx, double dy, double dz,
                        double *out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (long q = 0; q < count; ++q)
        oracle_newell_at(ijk[3 * q] * dx, ijk[3 * q + 1] * dy, ijk[3 * q + 2] * dz,
                         dx, dy, dz, out + 6 * q);
}
