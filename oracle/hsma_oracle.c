/*
 * HSMA oracle -- plain, slow, FP64 CPU implementation of the harmonic surface
 * mapping algorithm (Zhao, Liang & Xu, "Harmonic surface mapping algorithm
 * for fast electrostatic sums", arXiv:1806.04801).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.  Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * load it.  It shares no source, header, table or helper with the CUDA path.
 *
 * Every routine is written from the paper's definitions in plain loops; the
 * Python module oracle/hsma.py composes them into the algorithm in the order
 * the paper gives (Sec. II.C, "preparation" then "update").
 *
 * Conventions (Gaussian units): potential of charge q at distance d is q/d,
 * field E = -grad(phi), energy U = 1/2 sum_i q_i phi'(r_i) where phi' omits
 * the singular self term, force F_i = q_i E'(r_i).
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Image shells.  A source inside the box [-L/2, L/2) moved by k*L has        */
/* |x + kL| >= |k| L - L/2, so it can be inside the sphere of radius Rs only  */
/* when |k| < Rs/L + 1/2 (Eq. for the periodic sum and Eq. "diel").           */
/* ------------------------------------------------------------------------ */
int hsmo_num_shells(double Rs, double La)
{
    int k = 0;
    while ((k + 1) * La - 0.5 * La < Rs) ++k;
    return k;
}

/* ------------------------------------------------------------------------ */
/* In-set of Sec. II.A: all sources and images with |r| < Rs.                 */
/*   bc = 0 (periodic):  image of r_j under shift k is r_j + k∘L, charge q_j  */
/*   bc = 1 (grounded, the conducting limit gamma = -1 of Eq. "diel"):        */
/*          image is (-1)^k ∘ r_j + k∘L with charge (-1)^{|k|} q_j            */
/* Positions c are centred on the box (box = prod [-L_a/2, L_a/2)).           */
/* Order: shift k = 0 first (the N sources themselves, in input order), then  */
/* the other shifts in lexicographic order of (kx, ky, kz), each over j.      */
/* Returns the in-set size, or -1 if it would exceed cap.                     */
/* ------------------------------------------------------------------------ */
long hsmo_inset(long n, const double *c, const double *q, const double L[3], int bc,
                double Rs, long cap, double *out_xyz, double *out_q, long *out_src,
                int *out_shift)
{
    int K[3];
    for (int a = 0; a < 3; ++a) K[a] = hsmo_num_shells(Rs, L[a]);
    long m = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int kx = -K[0]; kx <= K[0]; ++kx)
            for (int ky = -K[1]; ky <= K[1]; ++ky)
                for (int kz = -K[2]; kz <= K[2]; ++kz) {
                    int zero = (kx == 0 && ky == 0 && kz == 0);
                    if ((pass == 0) != zero) continue;
                    int k[3] = {kx, ky, kz};
                    for (long j = 0; j < n; ++j) {
                        double p[3];
                        double qq = q[j];
                        for (int a = 0; a < 3; ++a) {
                            double s = 1.0;
                            if (bc == 1 && (abs(k[a]) % 2) == 1) s = -1.0;
                            p[a] = s * c[3 * j + a] + k[a] * L[a];
                        }
                        if (bc == 1 && ((abs(kx) + abs(ky) + abs(kz)) % 2) == 1) qq = -qq;
                        double r2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
                        if (!zero && !(r2 < Rs * Rs)) continue;
                        if (m >= cap) return -1;
                        for (int a = 0; a < 3; ++a) out_xyz[3 * m + a] = p[a];
                        out_q[m] = qq;
                        if (out_src) out_src[m] = j;
                        if (out_shift)
                            for (int a = 0; a < 3; ++a) out_shift[3 * m + a] = k[a];
                        ++m;
                    }
                }
    }
    return m;
}

/* ------------------------------------------------------------------------ */
/* Coulomb sums (the Phi_in of Sec. II.A and the point-image form of         */
/* Sec. II.B):  pot[t] = sum_s q_s / |x_t - y_s|,                            */
/*              field[t] = sum_s q_s (x_t - y_s) / |x_t - y_s|^3.            */
/* tskip[t] (optional) names one source index that target t skips (its own  */
/* copy).  Any other source at distance exactly zero is not skipped, so a     */
/* coincidence shows up as a non-finite result.                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    long ns, t0, t1;
    const double *sxyz, *sq, *txyz;
    const long *tskip;
    double *pot, *field;
} coul_job;

static void *coul_worker(void *arg)
{
    coul_job *J = (coul_job *)arg;
    for (long t = J->t0; t < J->t1; ++t) {
        double tx = J->txyz[3 * t], ty = J->txyz[3 * t + 1], tz = J->txyz[3 * t + 2];
        long skip = J->tskip ? J->tskip[t] : -1;
        double phi = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
        for (long s = 0; s < J->ns; ++s) {
            if (s == skip) continue;
            double dx = tx - J->sxyz[3 * s];
            double dy = ty - J->sxyz[3 * s + 1];
            double dz = tz - J->sxyz[3 * s + 2];
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            double qs = J->sq[s];
            phi += qs / d;
            if (J->field) {
                double w = qs / (d * d * d);
                ex += w * dx;
                ey += w * dy;
                ez += w * dz;
            }
        }
        J->pot[t] = phi;
        if (J->field) {
            J->field[3 * t] = ex;
            J->field[3 * t + 1] = ey;
            J->field[3 * t + 2] = ez;
        }
    }
    return NULL;
}

void hsmo_coulomb(long ns, const double *sxyz, const double *sq, long nt, const double *txyz,
                  const long *tskip, double *pot, double *field, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > nt) nthreads = (int)(nt > 0 ? nt : 1);
    pthread_t th[256];
    coul_job jobs[256];
    long per = (nt + nthreads - 1) / nthreads;
    for (int i = 0; i < nthreads; ++i) {
        coul_job j = {ns, i * per, (i + 1) * per < nt ? (i + 1) * per : nt,
                      sxyz, sq, txyz, tskip, pot, field};
        if (j.t0 > nt) j.t0 = nt;
        jobs[i] = j;
    }
    if (nthreads == 1) {
        coul_worker(&jobs[0]);
        return;
    }
    for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, coul_worker, &jobs[i]);
    for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
}

/* ------------------------------------------------------------------------ */
/* Harmonic basis of Eq. "harmonic": B_n^m = r^n Y_n^m, here in a real form   */
/* chosen for this oracle (any invertible change of basis within the span of  */
/* degree <= P leaves the least-squares fit unchanged):                       */
/*   index k = n^2 + n + m,  rho = |x| / Rs,  t = cos(theta), phi = azimuth   */
/*   m = 0 :  rho^n P_n(t)                                                    */
/*   m > 0 :  rho^n P_n^m(t) cos(m phi)                                       */
/*   m < 0 :  rho^n P_n^|m|(t) sin(|m| phi)                                   */
/* with P_n^m the associated Legendre functions WITHOUT the Condon-Shortley   */
/* phase and without normalisation, from the standard three-term recurrence   */
/* in the degree.                                                            */
/* ------------------------------------------------------------------------ */
void hsmo_basis(long np, const double *pts, int P, double Rs, double *out)
{
    int nb = (P + 1) * (P + 1);
    double *Pl = (double *)malloc(sizeof(double) * (P + 1) * (P + 1));
    for (long i = 0; i < np; ++i) {
        double x = pts[3 * i] / Rs, y = pts[3 * i + 1] / Rs, z = pts[3 * i + 2] / Rs;
        double r = sqrt(x * x + y * y + z * z);
        double *o = out + i * nb;
        if (r == 0.0) {
            for (int k = 0; k < nb; ++k) o[k] = 0.0;
            o[0] = 1.0;
            continue;
        }
        double t = z / r;
        double s = sqrt(fmax(0.0, 1.0 - t * t));
        double phi = atan2(y, x);
#define PL(nn, mm) Pl[(nn) * (P + 1) + (mm)]
        PL(0, 0) = 1.0;
        for (int m = 1; m <= P; ++m) PL(m, m) = (2.0 * m - 1.0) * s * PL(m - 1, m - 1);
        for (int m = 0; m < P; ++m) PL(m + 1, m) = (2.0 * m + 1.0) * t * PL(m, m);
        for (int m = 0; m <= P; ++m)
            for (int nn = m + 2; nn <= P; ++nn)
                PL(nn, m) = ((2.0 * nn - 1.0) * t * PL(nn - 1, m) - (nn + m - 1.0) * PL(nn - 2, m)) /
                            (double)(nn - m);
        double rn = 1.0;
        for (int nn = 0; nn <= P; ++nn) {
            for (int m = -nn; m <= nn; ++m) {
                int k = nn * nn + nn + m;
                if (m == 0)
                    o[k] = rn * PL(nn, 0);
                else if (m > 0)
                    o[k] = rn * PL(nn, m) * cos(m * phi);
                else
                    o[k] = rn * PL(nn, -m) * sin(-m * phi);
            }
            rn *= r;
        }
#undef PL
    }
    free(Pl);
}

/* ------------------------------------------------------------------------ */
/* Discrete least squares of Sec. II.A: x = argmin ||A x - b||_2 for a tall   */
/* m x n matrix A (row-major), by Householder QR of the column-equilibrated   */
/* matrix followed by back substitution.  Returns 0, or -1 if a column is     */
/* numerically zero (rank deficient).  rdiag (optional, n) receives |R_jj|.   */
/* ------------------------------------------------------------------------ */
int hsmo_lstsq(long m, long n, const double *A, const double *b, double *x, double *rdiag)
{
    if (m < n) return -1;
    double *W = (double *)malloc(sizeof(double) * m * n); /* column-major */
    double *y = (double *)malloc(sizeof(double) * m);
    double *scale = (double *)malloc(sizeof(double) * n);
    double *diag = (double *)malloc(sizeof(double) * n);
    int status = 0;
    for (long k = 0; k < n; ++k) {
        double s2 = 0.0;
        for (long i = 0; i < m; ++i) s2 += A[i * n + k] * A[i * n + k];
        double s = sqrt(s2);
        if (s == 0.0) { status = -1; goto done; }
        scale[k] = 1.0 / s;
        for (long i = 0; i < m; ++i) W[k * m + i] = A[i * n + k] * scale[k];
    }
    for (long i = 0; i < m; ++i) y[i] = b[i];
    for (long j = 0; j < n; ++j) {
        double *v = W + j * m; /* v lives in column j, rows j..m-1 */
        double nrm2 = 0.0;
        for (long i = j; i < m; ++i) nrm2 += v[i] * v[i];
        double nrm = sqrt(nrm2);
        if (nrm == 0.0) { status = -1; goto done; }
        double alpha = v[j] > 0.0 ? -nrm : nrm;
        v[j] -= alpha;
        double vv = 0.0;
        for (long i = j; i < m; ++i) vv += v[i] * v[i];
        for (long c = j + 1; c < n; ++c) {
            double *w = W + c * m;
            double d = 0.0;
            for (long i = j; i < m; ++i) d += v[i] * w[i];
            double tau = 2.0 * d / vv;
            for (long i = j; i < m; ++i) w[i] -= tau * v[i];
        }
        double d = 0.0;
        for (long i = j; i < m; ++i) d += v[i] * y[i];
        double tau = 2.0 * d / vv;
        for (long i = j; i < m; ++i) y[i] -= tau * v[i];
        diag[j] = alpha;
    }
    /* back substitution with R (upper triangle of W above the diagonal, diag) */
    for (long j = n - 1; j >= 0; --j) {
        double s = y[j];
        for (long c = j + 1; c < n; ++c) s -= W[c * m + j] * x[c];
        x[j] = s / diag[j];
    }
    for (long j = 0; j < n; ++j) x[j] *= scale[j];
    if (rdiag)
        for (long j = 0; j < n; ++j) rdiag[j] = fabs(diag[j]);
done:
    free(W);
    free(y);
    free(scale);
    free(diag);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Monitoring points on the circumsphere for the periodic case (Sec. II.A,   */
/* Fibonacci grid): for i = 1..Nm, latitude asin((2i-1)/Nm - 1) and azimuth  */
/* 2 pi i w with w = (sqrt 5 - 1)/2.  The printed "polar angle" is read as a */
/* latitude, which spreads the points over the whole sphere.                 */
/* ------------------------------------------------------------------------ */
void hsmo_monitor_sphere(int nm, double R0, double *out)
{
    double w = (sqrt(5.0) - 1.0) / 2.0;
    for (int i = 1; i <= nm; ++i) {
        double zu = (2.0 * i - 1.0) / nm - 1.0; /* sin(latitude) */
        double lat = asin(zu);
        double az = 2.0 * M_PI * i * w;
        double *o = out + 3 * (i - 1);
        o[0] = R0 * cos(lat) * cos(az);
        o[1] = R0 * cos(lat) * sin(az);
        o[2] = R0 * sin(lat);
    }
}

/* Periodic partner x~ = x - k L of a monitoring point, with k chosen so that */
/* x~ lies in the central box: k_a = round(x_a / L_a), ties away from zero.    */
void hsmo_wrap_into_box(long np, const double *pts, const double L[3], double *out)
{
    for (long i = 0; i < np; ++i)
        for (int a = 0; a < 3; ++a) {
            double k = round(pts[3 * i + a] / L[a]);
            out[3 * i + a] = pts[3 * i + a] - k * L[a];
        }
}

/* ------------------------------------------------------------------------ */
/* Monitoring points on the box boundary for non-periodic conditions         */
/* (Sec. II.A: "nearly uniformly distributed on the boundary").  The paper   */
/* gives no recipe; this oracle reads it as: K points split over the six     */
/* faces in proportion to face area (largest remainder, ties to the lower    */
/* face), and on a face with n points the i-th point (i = 0..n-1) sits at    */
/* unit-square coordinates ((i + 1/2)/n, frac(i w + 1/2)), w = (sqrt5-1)/2.   */
/* Face order: -x, +x, -y, +y, -z, +z; (u, v) span the two other axes in      */
/* increasing axis order.  Returns the number of points written (= K).       */
/* ------------------------------------------------------------------------ */
int hsmo_monitor_faces(int K, const double L[3], double *out)
{
    double area[6];
    for (int f = 0; f < 6; ++f) {
        int a = f / 2;
        area[f] = L[(a + 1) % 3] * L[(a + 2) % 3];
    }
    double tot = 0.0;
    for (int f = 0; f < 6; ++f) tot += area[f];
    int cnt[6], used = 0;
    double frac[6];
    for (int f = 0; f < 6; ++f) {
        double quota = K * area[f] / tot;
        cnt[f] = (int)floor(quota);
        frac[f] = quota - cnt[f];
        used += cnt[f];
    }
    while (used < K) {
        int best = 0;
        for (int f = 1; f < 6; ++f)
            if (frac[f] > frac[best]) best = f;
        cnt[best] += 1;
        frac[best] = -1.0;
        ++used;
    }
    double w = (sqrt(5.0) - 1.0) / 2.0;
    int o = 0;
    for (int f = 0; f < 6; ++f) {
        int a = f / 2;
        double side = (f % 2 == 0) ? -0.5 : 0.5;
        int ua = (a == 0) ? 1 : 0;
        int va = (a == 2) ? 1 : 2;
        for (int i = 0; i < cnt[f]; ++i) {
            double u = (i + 0.5) / cnt[f];
            double v = fmod(i * w + 0.5, 1.0);
            double p[3];
            p[a] = side * L[a];
            p[ua] = (u - 0.5) * L[ua];
            p[va] = (v - 0.5) * L[va];
            for (int b = 0; b < 3; ++b) out[3 * o + b] = p[b];
            ++o;
        }
    }
    return o;
}

/* ------------------------------------------------------------------------ */
/* Fibonacci numerical integration on a sphere (Sec. II.B):                  */
/*   int f dS ~ (2 pi R^2 / F2) sum_{j=0}^{F2} [1 + cos(pi z_j)]             */
/*               [f(R, th_j, ph_j) + f(R, th_j, pi + ph_j)],                 */
/*   z_j = -1 + 2j/F2,  th_j = acos(z_j + sin(pi z_j)/pi),  ph_j = pi j F1/F2. */
/* Writes 2(F2+1) unit directions (node 2j then 2j+1) and their weights for  */
/* a sphere of radius R.                                                     */
/* ------------------------------------------------------------------------ */
void hsmo_quadrature(int F2, int F1, double R, double *dirs, double *w)
{
    for (int j = 0; j <= F2; ++j) {
        double zj = -1.0 + 2.0 * j / F2;
        double ct = zj + sin(M_PI * zj) / M_PI;
        if (ct > 1.0) ct = 1.0;
        if (ct < -1.0) ct = -1.0;
        double th = acos(ct);
        double ph = M_PI * (double)j * (double)F1 / (double)F2;
        double wj = 2.0 * M_PI * R * R / F2 * (1.0 + cos(M_PI * zj));
        for (int h = 0; h < 2; ++h) {
            double p = ph + h * M_PI;
            double *d = dirs + 3 * (2 * j + h);
            d[0] = sin(th) * cos(p);
            d[1] = sin(th) * sin(p);
            d[2] = cos(th);
            w[2 * j + h] = wj;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Ewald summation for a neutral periodic cell (independent check of the     */
/* periodic sum of Sec. II; conducting "tinfoil" surroundings, i.e. no dipole */
/* surface term).  Rectangular cell L[0..2].  For each charge i:              */
/*  pot[i]   = sum_j sum_n' q_j erfc(beta d)/d                                */
/*           + (4 pi / V) sum_{k != 0} exp(-k^2/4beta^2)/k^2 sum_j q_j cos(k.(r_i - r_j)) */
/*           - 2 beta q_i / sqrt(pi)                                          */
/*  field[i] = -grad_i of the same (excluding the i = j, n = 0 term).         */
/* The real-space sum runs over |n_a| <= nreal cells, the reciprocal sum over */
/* integer vectors with |m_a| <= kmax.                                        */
/* ------------------------------------------------------------------------ */
void hsmo_ewald(long n, const double *xyz, const double *q, const double L[3], double beta,
                int nreal, int kmax, double *pot, double *field)
{
    double V = L[0] * L[1] * L[2];
    for (long i = 0; i < n; ++i) {
        double phi = 0.0, e[3] = {0.0, 0.0, 0.0};
        for (long j = 0; j < n; ++j)
            for (int nx = -nreal; nx <= nreal; ++nx)
                for (int ny = -nreal; ny <= nreal; ++ny)
                    for (int nz = -nreal; nz <= nreal; ++nz) {
                        if (i == j && nx == 0 && ny == 0 && nz == 0) continue;
                        double d[3] = {xyz[3 * i] - xyz[3 * j] - nx * L[0],
                                       xyz[3 * i + 1] - xyz[3 * j + 1] - ny * L[1],
                                       xyz[3 * i + 2] - xyz[3 * j + 2] - nz * L[2]};
                        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                        double ec = erfc(beta * r);
                        phi += q[j] * ec / r;
                        double g = q[j] * (ec + 2.0 * beta * r / sqrt(M_PI) * exp(-beta * beta * r * r)) /
                                   (r * r * r);
                        for (int a = 0; a < 3; ++a) e[a] += g * d[a];
                    }
        for (int mx = -kmax; mx <= kmax; ++mx)
            for (int my = -kmax; my <= kmax; ++my)
                for (int mz = -kmax; mz <= kmax; ++mz) {
                    if (mx == 0 && my == 0 && mz == 0) continue;
                    double k[3] = {2.0 * M_PI * mx / L[0], 2.0 * M_PI * my / L[1], 2.0 * M_PI * mz / L[2]};
                    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                    double f = 4.0 * M_PI / V * exp(-k2 / (4.0 * beta * beta)) / k2;
                    double cs = 0.0, sn = 0.0;
                    for (long j = 0; j < n; ++j) {
                        double arg = k[0] * (xyz[3 * i] - xyz[3 * j]) + k[1] * (xyz[3 * i + 1] - xyz[3 * j + 1]) +
                                     k[2] * (xyz[3 * i + 2] - xyz[3 * j + 2]);
                        cs += q[j] * cos(arg);
                        sn += q[j] * sin(arg);
                    }
                    phi += f * cs;
                    for (int a = 0; a < 3; ++a) e[a] += f * k[a] * sn;
                }
        phi -= 2.0 * beta * q[i] / sqrt(M_PI);
        pot[i] = phi;
        if (field)
            for (int a = 0; a < 3; ++a) field[3 * i + a] = e[a];
    }
}

/* ------------------------------------------------------------------------ */
/* The same Ewald sum as hsmo_ewald, with the reciprocal part through        */
/* structure factors S(k) = sum_j q_j exp(i k.r_j) (O(N K) instead of        */
/* O(N^2 K)) and the real part over |n_a| <= nreal cells; for larger checks. */
/* ------------------------------------------------------------------------ */
void hsmo_ewald_sf(long n, const double *xyz, const double *q, const double L[3], double beta, int nreal,
                   int kmax, double *pot, double *field)
{
    double V = L[0] * L[1] * L[2];
    for (long i = 0; i < n; ++i) {
        double phi = 0.0, e[3] = {0.0, 0.0, 0.0};
        for (long j = 0; j < n; ++j)
            for (int nx = -nreal; nx <= nreal; ++nx)
                for (int ny = -nreal; ny <= nreal; ++ny)
                    for (int nz = -nreal; nz <= nreal; ++nz) {
                        if (i == j && nx == 0 && ny == 0 && nz == 0) continue;
                        double d[3] = {xyz[3 * i] - xyz[3 * j] - nx * L[0],
                                       xyz[3 * i + 1] - xyz[3 * j + 1] - ny * L[1],
                                       xyz[3 * i + 2] - xyz[3 * j + 2] - nz * L[2]};
                        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                        if (beta * r > 7.0) continue; /* erfc(7) ~ 4e-23 */
                        double ec = erfc(beta * r);
                        phi += q[j] * ec / r;
                        double g = q[j] * (ec + 2.0 * beta * r / sqrt(M_PI) * exp(-beta * beta * r * r)) /
                                   (r * r * r);
                        for (int a = 0; a < 3; ++a) e[a] += g * d[a];
                    }
        pot[i] = phi - 2.0 * beta * q[i] / sqrt(M_PI);
        if (field)
            for (int a = 0; a < 3; ++a) field[3 * i + a] = e[a];
    }
    double *c = (double *)malloc(sizeof(double) * n), *s = (double *)malloc(sizeof(double) * n);
    for (int mx = -kmax; mx <= kmax; ++mx)
        for (int my = -kmax; my <= kmax; ++my)
            for (int mz = -kmax; mz <= kmax; ++mz) {
                if (mx == 0 && my == 0 && mz == 0) continue;
                double k[3] = {2.0 * M_PI * mx / L[0], 2.0 * M_PI * my / L[1], 2.0 * M_PI * mz / L[2]};
                double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                double f = 4.0 * M_PI / V * exp(-k2 / (4.0 * beta * beta)) / k2;
                if (f < 1e-300) continue;
                double Sc = 0.0, Ss = 0.0;
                for (long j = 0; j < n; ++j) {
                    double arg = k[0] * xyz[3 * j] + k[1] * xyz[3 * j + 1] + k[2] * xyz[3 * j + 2];
                    c[j] = cos(arg);
                    s[j] = sin(arg);
                    Sc += q[j] * c[j];
                    Ss += q[j] * s[j];
                }
                for (long i = 0; i < n; ++i) {
                    /* sum_j q_j cos(k.(r_i - r_j)) = c_i Sc + s_i Ss; the sin form for the field */
                    pot[i] += f * (c[i] * Sc + s[i] * Ss);
                    if (field) {
                        double sn = s[i] * Sc - c[i] * Ss;
                        for (int a = 0; a < 3; ++a) field[3 * i + a] += f * k[a] * sn;
                    }
                }
            }
    free(c);
    free(s);
}

/* ------------------------------------------------------------------------ */
/* Ewald sum for large periodic systems (tinfoil, neutral): the real-space    */
/* part over pairs closer than rc (minimum image; rc < L_a / 2, cell lists    */
/* of at least 3 cells per axis), the reciprocal part over |k| <= kcut        */
/* through structure factors S(k) = sum_j q_j exp(i k.r_j), the self term     */
/* -beta q_i / sqrt(pi).  Returns the energy                                  */
/*   U = 1/2 sum_i sum_(j,n)' q_i q_j erfc(beta r)/r                           */
/*     + (2 pi / V) sum_(k != 0) exp(-k^2 / 4 beta^2) / k^2 |S(k)|^2          */
/*     - beta / sqrt(pi) sum_i q_i^2,                                         */
/* and the potential (self term removed) and field at the npick particles    */
/* pick[] (want_energy = 0: only these; the real-space energy, O(N^2 rc^3), */
/* is skipped and 0 returned).  A check of the large-N study of Sec. III,    */
/* independent of HSMA.                                                      */
/* Threads split the particles; their partial sums are added in thread order  */
/* (deterministic for a given thread count).                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    long n, i0, i1;
    const double *xyz, *q;
    double L[3], beta, rc;
    int nc[3];
    const long *head, *next;
    int M[3];
    double kcut;
    double *Sre, *Sim; /* this thread's partial structure factors, (2M+1)^3 */
    double ureal;
    int want_energy;   /* 0: skip the real-space energy (picked particles only) */
} ewc_job;

static long ewc_cell(const double *p, const double L[3], const int nc[3])
{
    int c[3];
    for (int a = 0; a < 3; ++a) {
        double f = p[a] / L[a];
        f -= floor(f);
        int k = (int)(f * nc[a]);
        c[a] = k >= nc[a] ? nc[a] - 1 : k;
    }
    return ((long)c[0] * nc[1] + c[1]) * nc[2] + c[2];
}

/* real-space potential and field at point p (excluding particle `self`) */
static void ewc_real_at(const ewc_job *J, const double *p, long self, double *phi, double *e)
{
    int c[3];
    for (int a = 0; a < 3; ++a) {
        double f = p[a] / J->L[a];
        f -= floor(f);
        int k = (int)(f * J->nc[a]);
        c[a] = k >= J->nc[a] ? J->nc[a] - 1 : k;
    }
    double ph = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
    const double rc2 = J->rc * J->rc, b = J->beta, tsp = 2.0 * J->beta / sqrt(M_PI);
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                int cc[3] = {(c[0] + dx + J->nc[0]) % J->nc[0], (c[1] + dy + J->nc[1]) % J->nc[1],
                             (c[2] + dz + J->nc[2]) % J->nc[2]};
                long cell = ((long)cc[0] * J->nc[1] + cc[1]) * J->nc[2] + cc[2];
                for (long j = J->head[cell]; j >= 0; j = J->next[j]) {
                    if (j == self) continue;
                    double d[3];
                    for (int a = 0; a < 3; ++a) {
                        double v = p[a] - J->xyz[3 * j + a];
                        v -= J->L[a] * floor(v / J->L[a] + 0.5); /* minimum image */
                        d[a] = v;
                    }
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 >= rc2) continue;
                    double r = sqrt(r2);
                    double ec = erfc(b * r);
                    ph += J->q[j] * ec / r;
                    if (e) {
                        double g = J->q[j] * (ec + tsp * r * exp(-b * b * r2)) / (r2 * r);
                        ex += g * d[0];
                        ey += g * d[1];
                        ez += g * d[2];
                    }
                }
            }
    *phi = ph;
    if (e) {
        e[0] = ex;
        e[1] = ey;
        e[2] = ez;
    }
}

/* Each thread: the real-space energy of its particles, and their partial   */
/* structure factors, particles taken in blocks of EWC_B so that S(k) is     */
/* traversed once per block.                                                 */
#define EWC_B 128
static void *ewc_worker(void *arg)
{
    ewc_job *J = (ewc_job *)arg;
    const int Mx = J->M[0], My = J->M[1], Mz = J->M[2];
    const int wx = 2 * Mx + 1, wy = 2 * My + 1, wz = 2 * Mz + 1;
    const long sy = wz, sx = (long)wy * sy;
    /* per block: cos/sin of 2 pi m x_a / L_a, [m][particle] */
    double *cx = (double *)malloc(sizeof(double) * wx * EWC_B), *sxn = (double *)malloc(sizeof(double) * wx * EWC_B);
    double *cy = (double *)malloc(sizeof(double) * wy * EWC_B), *syn = (double *)malloc(sizeof(double) * wy * EWC_B);
    double *cz = (double *)malloc(sizeof(double) * wz * EWC_B), *szn = (double *)malloc(sizeof(double) * wz * EWC_B);
    double pr[EWC_B], pim[EWC_B];
    const double kc2 = J->kcut * J->kcut;
    double ureal = 0.0;
    for (long b0 = J->i0; b0 < J->i1; b0 += EWC_B) {
        const int nb = (int)(J->i1 - b0 < EWC_B ? J->i1 - b0 : EWC_B);
        for (int u = 0; u < nb; ++u) {
            const long i = b0 + u;
            const double *p = J->xyz + 3 * i;
            if (J->want_energy) {
                double phi;
                ewc_real_at(J, p, i, &phi, NULL);
                ureal += J->q[i] * phi;
            }
            for (int m = -Mx; m <= Mx; ++m) {
                double t = 2.0 * M_PI * m * p[0] / J->L[0];
                cx[(m + Mx) * EWC_B + u] = cos(t);
                sxn[(m + Mx) * EWC_B + u] = sin(t);
            }
            for (int m = -My; m <= My; ++m) {
                double t = 2.0 * M_PI * m * p[1] / J->L[1];
                cy[(m + My) * EWC_B + u] = cos(t);
                syn[(m + My) * EWC_B + u] = sin(t);
            }
            for (int m = -Mz; m <= Mz; ++m) {
                double t = 2.0 * M_PI * m * p[2] / J->L[2];
                cz[(m + Mz) * EWC_B + u] = cos(t);
                szn[(m + Mz) * EWC_B + u] = sin(t);
            }
        }
        for (int mx = -Mx; mx <= Mx; ++mx) {
            double kx = 2.0 * M_PI * mx / J->L[0];
            if (kx * kx > kc2) continue;
            for (int my = -My; my <= My; ++my) {
                double ky = 2.0 * M_PI * my / J->L[1];
                double rem = kc2 - kx * kx - ky * ky;
                if (rem < 0.0) continue;
                int mz1 = (int)floor(sqrt(rem) * J->L[2] / (2.0 * M_PI));
                if (mz1 > Mz) mz1 = Mz;
                const double *ax = cx + (mx + Mx) * EWC_B, *bx = sxn + (mx + Mx) * EWC_B;
                const double *ay = cy + (my + My) * EWC_B, *by = syn + (my + My) * EWC_B;
                for (int u = 0; u < nb; ++u) {
                    const double qi = J->q[b0 + u];
                    pr[u] = qi * (ax[u] * ay[u] - bx[u] * by[u]);
                    pim[u] = qi * (ax[u] * by[u] + bx[u] * ay[u]);
                }
                const long base = (long)(mx + Mx) * sx + (long)(my + My) * sy + Mz;
                for (int mz = -mz1; mz <= mz1; ++mz) {
                    const double *c = cz + (mz + Mz) * EWC_B, *sn = szn + (mz + Mz) * EWC_B;
                    double re = 0.0, im = 0.0;
                    for (int u = 0; u < nb; ++u) {
                        re += pr[u] * c[u] - pim[u] * sn[u];
                        im += pr[u] * sn[u] + pim[u] * c[u];
                    }
                    J->Sre[base + mz] += re;
                    J->Sim[base + mz] += im;
                }
            }
        }
    }
    J->ureal = 0.5 * ureal;
    free(cx);
    free(sxn);
    free(cy);
    free(syn);
    free(cz);
    free(szn);
    return NULL;
}

double hsmo_ewald_cells(long n, const double *xyz, const double *q, const double L[3], double beta, double rc,
                        double kcut, int nthreads, int want_energy, long npick, const long *pick, double *pick_pot,
                        double *pick_field)
{
    int nc[3], M[3];
    for (int a = 0; a < 3; ++a) {
        nc[a] = (int)floor(L[a] / rc);
        if (nc[a] < 3 || 2.0 * rc >= L[a]) return NAN; /* cell lists need 3 cells, minimum image rc < L/2 */
        M[a] = (int)ceil(kcut * L[a] / (2.0 * M_PI));
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > n) nthreads = (int)(n > 0 ? n : 1);
    const long ncell = (long)nc[0] * nc[1] * nc[2];
    long *head = (long *)malloc(sizeof(long) * ncell), *next = (long *)malloc(sizeof(long) * n);
    for (long c = 0; c < ncell; ++c) head[c] = -1;
    for (long j = n - 1; j >= 0; --j) {
        long c = ewc_cell(xyz + 3 * j, L, nc);
        next[j] = head[c];
        head[c] = j;
    }
    const long nk = (long)(2 * M[0] + 1) * (2 * M[1] + 1) * (2 * M[2] + 1);
    ewc_job jobs[256];
    pthread_t th[256];
    long per = (n + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        ewc_job *J = &jobs[t];
        J->n = n;
        J->i0 = t * per < n ? t * per : n;
        J->i1 = (t + 1) * per < n ? (t + 1) * per : n;
        J->xyz = xyz;
        J->q = q;
        for (int a = 0; a < 3; ++a) {
            J->L[a] = L[a];
            J->nc[a] = nc[a];
            J->M[a] = M[a];
        }
        J->beta = beta;
        J->rc = rc;
        J->head = head;
        J->next = next;
        J->kcut = kcut;
        J->Sre = (double *)calloc(nk, sizeof(double));
        J->Sim = (double *)calloc(nk, sizeof(double));
        J->ureal = 0.0;
        J->want_energy = want_energy;
    }
    if (nthreads == 1)
        ewc_worker(&jobs[0]);
    else {
        for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, ewc_worker, &jobs[t]);
        for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    }
    /* structure factors and real-space energy, added in thread order */
    double *Sre = jobs[0].Sre, *Sim = jobs[0].Sim;
    double ureal = jobs[0].ureal;
    for (int t = 1; t < nthreads; ++t) {
        for (long k = 0; k < nk; ++k) {
            Sre[k] += jobs[t].Sre[k];
            Sim[k] += jobs[t].Sim[k];
        }
        ureal += jobs[t].ureal;
        free(jobs[t].Sre);
        free(jobs[t].Sim);
    }
    const double V = L[0] * L[1] * L[2], kc2 = kcut * kcut;
    const long sy = 2 * M[2] + 1, sx = (2 * M[1] + 1) * sy;
    double urec = 0.0, q2 = 0.0;
    for (int mx = -M[0]; mx <= M[0]; ++mx)
        for (int my = -M[1]; my <= M[1]; ++my)
            for (int mz = -M[2]; mz <= M[2]; ++mz) {
                if (mx == 0 && my == 0 && mz == 0) continue;
                double k[3] = {2.0 * M_PI * mx / L[0], 2.0 * M_PI * my / L[1], 2.0 * M_PI * mz / L[2]};
                double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                if (k2 > kc2) continue;
                long idx = (long)(mx + M[0]) * sx + (long)(my + M[1]) * sy + (mz + M[2]);
                urec += exp(-k2 / (4.0 * beta * beta)) / k2 * (Sre[idx] * Sre[idx] + Sim[idx] * Sim[idx]);
            }
    urec *= 2.0 * M_PI / V;
    for (long i = 0; i < n; ++i) q2 += q[i] * q[i];
    const double energy = want_energy ? ureal + urec - beta / sqrt(M_PI) * q2 : 0.0;
    /* potential and field at the picked particles */
    for (long s = 0; s < npick; ++s) {
        long i = pick[s];
        const double *p = xyz + 3 * i;
        double phi, e[3];
        ewc_real_at(&jobs[0], p, i, &phi, e);
        for (int mx = -M[0]; mx <= M[0]; ++mx)
            for (int my = -M[1]; my <= M[1]; ++my)
                for (int mz = -M[2]; mz <= M[2]; ++mz) {
                    if (mx == 0 && my == 0 && mz == 0) continue;
                    double k[3] = {2.0 * M_PI * mx / L[0], 2.0 * M_PI * my / L[1], 2.0 * M_PI * mz / L[2]};
                    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                    if (k2 > kc2) continue;
                    long idx = (long)(mx + M[0]) * sx + (long)(my + M[1]) * sy + (mz + M[2]);
                    double f = 4.0 * M_PI / V * exp(-k2 / (4.0 * beta * beta)) / k2;
                    double arg = k[0] * p[0] + k[1] * p[1] + k[2] * p[2];
                    double c = cos(arg), sn = sin(arg);
                    /* sum_j q_j cos(k.(r - r_j)) = Re(e^{ik.r} conj S);  sin form for the field */
                    phi += f * (c * Sre[idx] + sn * Sim[idx]);
                    double im = sn * Sre[idx] - c * Sim[idx];
                    for (int a = 0; a < 3; ++a) e[a] += f * k[a] * im;
                }
        pick_pot[s] = phi - 2.0 * beta * q[i] / sqrt(M_PI);
        for (int a = 0; a < 3; ++a) pick_field[3 * s + a] = e[a];
    }
    free(jobs[0].Sre);
    free(jobs[0].Sim);
    free(head);
    free(next);
    return energy;
}
