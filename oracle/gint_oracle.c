/*
 * Plain FP64 CPU oracle for the real-space grid integration of an LCAO (numerical atomic
 * orbital) Kohn-Sham code, written from the method's definitions:
 *
 *   basis     phi_mu(r) = f_{zeta l}(|r - tau_I|) Y_lm(r_hat)       (Sec. IV.A; radial times
 *             spherical harmonic, the form the paper gives for projectors and ABFs, Sec. II.A
 *             and Sec. IV.C)
 *   vlocal    V_mu,nu(R) = Sum_r phi_mu(r - tau_I) V(r) phi_nu(r - tau_J - R) dV
 *             (two-centre template of Sec. IV.B with a multiplicative local operator,
 *             evaluated on the uniform real-space grid as Sec. IV.B describes)
 *   density   rho(r) = Sum_R Sum_mu,nu rho_mu,nu(R) phi_mu phi_nu    (Eq. density_matrix and
 *             the sentence after it, Sec. IV.B)
 *   force     Pulay term of Eq. force_lcao (Sec. IV.D): derivative of
 *             L = Sum_blocks Sum rho_mu,nu(R) V_mu,nu(R) with respect to the atom positions
 *             through the basis functions only (V(r) held fixed).
 *   strain    derivative of the same L with respect to a homogeneous strain of cell, atoms
 *             and grid (the grid part of the stress of Eq. stress), V(r) grid values fixed.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the CUDA library: it
 * shares no code, header, table or helper with it.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  It is deliberately slow: a loop over grid
 * points, a brute-force search over all atoms and all periodic images for each point, and
 * a dense double loop over the orbitals found.  OpenMP (if enabled at build time) only
 * splits the grid points across threads; every thread accumulates privately and the
 * partial results are added in thread order.
 *
 * Conventions (readings of points the paper leaves open):
 *   - cell rows a1,a2,a3; grid point (i,j,k) at r = (i/N1) a1 + (j/N2) a2 + (k/N3) a3,
 *     linear index (i*N2 + j)*N3 + k; dV = |det A| / (N1 N2 N3).
 *   - tau is used as given (not wrapped into the cell); a block key (I, J, R) with
 *     R = n1 a1 + n2 a2 + n3 a3 couples phi centred at tau_I with phi centred at tau_J + R,
 *     and exists iff |tau_J + R - tau_I| < rc_I + rc_J.  Keys are sorted by (I, J, n1, n2, n3).
 *   - radial functions are clamped cubic splines through the tabulated f(r_i), r_i = i dr,
 *     with end slopes f'(0) (given) and f'(r_last) = 0; f = 0 for r >= rc.  The spline is
 *     built here in its second-derivative ("moment") form.
 *   - real harmonics without the Condon-Shortley phase, per l ordered m = 0, +1, -1, +2, -2;
 *     l = 1 is sqrt(3/4pi) (z, x, y)/r.
 *   - at r < 1e-12: phi = f(0) Y_00 for l = 0 and 0 otherwise; grad phi = f'(0) sqrt(3/4pi)
 *     e_m for l = 1 and 0 otherwise.
 *
 * Parity pins: see tests/test_oracle_pins.py (closed forms, quadrature, invariants, finite
 * differences).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXRAD 16
#define OR_MAXORB 64

typedef struct {
    int nrad, norb, ntab;
    double rcut, dr;
    int l[OR_MAXRAD];
    double *y;    /* [nrad][ntab] table values */
    double *m2;   /* [nrad][ntab] spline second derivatives */
} or_species;

typedef struct {
    double cell[9];      /* rows a1, a2, a3 */
    double g[9];         /* g[3*c + i]: component c of reciprocal vector g_i (a_i . g_j = delta_ij) */
    double gnorm[3];
    int grid[3];
    int64_t npts;
    double dV;
    int natoms, nspecies;
    int *spc;            /* [natoms] */
    double *tau;         /* [natoms*3] */
    or_species *sp;
    int *img_lo, *img_hi;   /* [natoms*3]: image ranges reaching the cell */
    /* block lookup (filled per call from the keys passed in) */
} or_ctx;

/* ------------------------------------------------------------------ spline (moment form) */
static void or_build_spline(const double *y, int n, double h, double d0, double dn, double *m)
{
    /* Clamped cubic spline: solve for second derivatives m_0..m_{n-1} at equally spaced
     * knots; tridiagonal system by the Thomas algorithm. */
    double *c = (double *)malloc(sizeof(double) * n);
    double *d = (double *)malloc(sizeof(double) * n);
    /* row 0: 2 m0 + m1 = 6/h ((y1-y0)/h - d0) */
    double b0 = 2.0, c0 = 1.0, r0 = 6.0 / h * ((y[1] - y[0]) / h - d0);
    c[0] = c0 / b0;
    d[0] = r0 / b0;
    for (int i = 1; i < n - 1; ++i) {
        double a = 1.0, b = 4.0, cc = 1.0;
        double r = 6.0 * (y[i + 1] - 2.0 * y[i] + y[i - 1]) / (h * h);
        double den = b - a * c[i - 1];
        c[i] = cc / den;
        d[i] = (r - a * d[i - 1]) / den;
    }
    {
        int i = n - 1;
        double a = 1.0, b = 2.0;
        double r = 6.0 / h * (dn - (y[n - 1] - y[n - 2]) / h);
        double den = b - a * c[i - 1];
        d[i] = (r - a * d[i - 1]) / den;
        c[i] = 0.0;
    }
    m[n - 1] = d[n - 1];
    for (int i = n - 2; i >= 0; --i) m[i] = d[i] - c[i] * m[i + 1];
    free(c);
    free(d);
}

/* value and derivative of radial `ir` of species `s` at r (0 beyond the cutoff) */
static double or_radial(const or_species *s, int ir, double r, double *dfdr)
{
    if (r >= s->rcut) {
        if (dfdr) *dfdr = 0.0;
        return 0.0;
    }
    const double h = s->dr;
    const double *y = s->y + (size_t)ir * s->ntab;
    const double *m = s->m2 + (size_t)ir * s->ntab;
    int i = (int)floor(r / h);
    if (i > s->ntab - 2) i = s->ntab - 2;
    if (i < 0) i = 0;
    double xl = i * h, xr = (i + 1) * h;
    double A = (xr - r) / h, B = (r - xl) / h;
    double v = A * y[i] + B * y[i + 1] + ((A * A * A - A) * m[i] + (B * B * B - B) * m[i + 1]) * h * h / 6.0;
    if (dfdr)
        *dfdr = (y[i + 1] - y[i]) / h - (3.0 * A * A - 1.0) / 6.0 * h * m[i] + (3.0 * B * B - 1.0) / 6.0 * h * m[i + 1];
    return v;
}

/* ------------------------------------------------------------------ real Y_lm on the unit sphere */
/* Y_lm as a polynomial in the unit vector u, and its gradient with respect to u (treating
 * the polynomial as a function on R^3).  Order per l: m = 0, +1, -1, +2, -2. */
static void or_ylm(int l, const double u[3], double *Y, double (*dY)[3])
{
    const double pi = acos(-1.0);
    double x = u[0], y = u[1], z = u[2];
    if (l == 0) {
        double c = 0.5 / sqrt(pi);
        Y[0] = c;
        if (dY) { dY[0][0] = dY[0][1] = dY[0][2] = 0.0; }
    } else if (l == 1) {
        double c = sqrt(3.0 / (4.0 * pi));
        Y[0] = c * z; Y[1] = c * x; Y[2] = c * y;
        if (dY) {
            memset(dY, 0, sizeof(double) * 9);
            dY[0][2] = c; dY[1][0] = c; dY[2][1] = c;
        }
    } else {
        double c0 = sqrt(5.0 / (16.0 * pi));
        double c1 = sqrt(15.0 / (4.0 * pi));
        double c2 = sqrt(15.0 / (16.0 * pi));
        Y[0] = c0 * (3.0 * z * z - 1.0);     /* on the unit sphere x^2+y^2+z^2 = 1 */
        Y[1] = c1 * x * z;
        Y[2] = c1 * y * z;
        Y[3] = c2 * (x * x - y * y);
        Y[4] = c1 * x * y;
        if (dY) {
            dY[0][0] = 0.0;        dY[0][1] = 0.0;         dY[0][2] = 6.0 * c0 * z;
            dY[1][0] = c1 * z;     dY[1][1] = 0.0;         dY[1][2] = c1 * x;
            dY[2][0] = 0.0;        dY[2][1] = c1 * z;      dY[2][2] = c1 * y;
            dY[3][0] = 2 * c2 * x; dY[3][1] = -2 * c2 * y; dY[3][2] = 0.0;
            dY[4][0] = c1 * y;     dY[4][1] = c1 * x;      dY[4][2] = 0.0;
        }
    }
}

/* all orbitals of species s at displacement d = r - centre; grad (nullable) is [norb][3],
 * the gradient with respect to r.  Returns the number of orbitals. */
static int or_phi(const or_species *s, const double d[3], double *phi, double *grad)
{
    const double pi = acos(-1.0);
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    int o = 0;
    for (int ir = 0; ir < s->nrad; ++ir) {
        int l = s->l[ir];
        int nm = 2 * l + 1;
        if (r >= s->rcut) {
            for (int m = 0; m < nm; ++m, ++o) {
                phi[o] = 0.0;
                if (grad) grad[3 * o] = grad[3 * o + 1] = grad[3 * o + 2] = 0.0;
            }
            continue;
        }
        if (r < 1e-12) {
            double df0;
            double f0 = or_radial(s, ir, 0.0, &df0);
            for (int m = 0; m < nm; ++m, ++o) {
                phi[o] = (l == 0) ? f0 * 0.5 / sqrt(pi) : 0.0;
                if (grad) {
                    grad[3 * o] = grad[3 * o + 1] = grad[3 * o + 2] = 0.0;
                    if (l == 1) {
                        /* m = 0 -> z, +1 -> x, -1 -> y */
                        int axis = (m == 0) ? 2 : (m == 1 ? 0 : 1);
                        grad[3 * o + axis] = df0 * sqrt(3.0 / (4.0 * pi));
                    }
                }
            }
            continue;
        }
        double u[3] = {d[0] / r, d[1] / r, d[2] / r};
        double df;
        double f = or_radial(s, ir, r, grad ? &df : NULL);
        double Y[5], dY[5][3];
        or_ylm(l, u, Y, grad ? dY : NULL);
        for (int m = 0; m < nm; ++m, ++o) {
            phi[o] = f * Y[m];
            if (grad) {
                /* grad [f(r) Y(u)] = f'(r) u Y + (f/r) (dY/du - (u . dY/du) u) */
                double ud = u[0] * dY[m][0] + u[1] * dY[m][1] + u[2] * dY[m][2];
                for (int c = 0; c < 3; ++c)
                    grad[3 * o + c] = df * u[c] * Y[m] + f / r * (dY[m][c] - ud * u[c]);
            }
        }
    }
    return o;
}

/* ------------------------------------------------------------------ context */
void oracle_free(or_ctx *c);

or_ctx *oracle_new(const double *cell, int natoms, const int *species, const double *tau,
                   int nspecies, const int *sp_nrad, const double *sp_rcut, const double *sp_dr,
                   const int *sp_ntab, const int *rad_l, const double *rad_dfdr0,
                   const double *ftab, const int *grid)
{
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    memcpy(c->cell, cell, sizeof(double) * 9);
    const double *A = cell;
    double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                 A[2] * (A[3] * A[7] - A[4] * A[6]);
    /* reciprocal vectors g_i = (a_j x a_k) / det */
    for (int i = 0; i < 3; ++i) {
        const double *aj = A + 3 * ((i + 1) % 3), *ak = A + 3 * ((i + 2) % 3);
        double gx = aj[1] * ak[2] - aj[2] * ak[1];
        double gy = aj[2] * ak[0] - aj[0] * ak[2];
        double gz = aj[0] * ak[1] - aj[1] * ak[0];
        c->g[0 + i] = gx / det;
        c->g[3 + i] = gy / det;
        c->g[6 + i] = gz / det;
        c->gnorm[i] = sqrt(gx * gx + gy * gy + gz * gz) / fabs(det);
    }
    for (int i = 0; i < 3; ++i) c->grid[i] = grid[i];
    c->npts = (int64_t)grid[0] * grid[1] * grid[2];
    c->dV = fabs(det) / (double)c->npts;
    c->natoms = natoms;
    c->nspecies = nspecies;
    c->spc = (int *)malloc(sizeof(int) * natoms);
    memcpy(c->spc, species, sizeof(int) * natoms);
    c->tau = (double *)malloc(sizeof(double) * 3 * natoms);
    memcpy(c->tau, tau, sizeof(double) * 3 * natoms);
    c->sp = (or_species *)calloc(nspecies, sizeof(or_species));
    int roff = 0;
    size_t toff = 0;
    for (int s = 0; s < nspecies; ++s) {
        or_species *S = &c->sp[s];
        S->nrad = sp_nrad[s];
        S->rcut = sp_rcut[s];
        S->dr = sp_dr[s];
        S->ntab = sp_ntab[s];
        S->norb = 0;
        S->y = (double *)malloc(sizeof(double) * S->nrad * S->ntab);
        S->m2 = (double *)malloc(sizeof(double) * S->nrad * S->ntab);
        for (int ir = 0; ir < S->nrad; ++ir) {
            S->l[ir] = rad_l[roff + ir];
            S->norb += 2 * S->l[ir] + 1;
            memcpy(S->y + (size_t)ir * S->ntab, ftab + toff, sizeof(double) * S->ntab);
            or_build_spline(S->y + (size_t)ir * S->ntab, S->ntab, S->dr, rad_dfdr0[roff + ir], 0.0,
                            S->m2 + (size_t)ir * S->ntab);
            toff += S->ntab;
        }
        roff += S->nrad;
    }
    /* image ranges: centre tau + n.A can reach a point with fractional coords in [0,1) */
    c->img_lo = (int *)malloc(sizeof(int) * 3 * natoms);
    c->img_hi = (int *)malloc(sizeof(int) * 3 * natoms);
    for (int I = 0; I < natoms; ++I) {
        const double *t = tau + 3 * I;
        double rc = c->sp[species[I]].rcut;
        for (int i = 0; i < 3; ++i) {
            double s = t[0] * c->g[0 + i] + t[1] * c->g[3 + i] + t[2] * c->g[6 + i];
            c->img_lo[3 * I + i] = (int)floor(-s - rc * c->gnorm[i]) - 1;
            c->img_hi[3 * I + i] = (int)ceil(1.0 - s + rc * c->gnorm[i]) + 1;
        }
    }
    return c;
}

void oracle_free(or_ctx *c)
{
    if (!c) return;
    for (int s = 0; s < c->nspecies; ++s) {
        free(c->sp[s].y);
        free(c->sp[s].m2);
    }
    free(c->sp);
    free(c->spc);
    free(c->tau);
    free(c->img_lo);
    free(c->img_hi);
    free(c);
}

double oracle_dV(const or_ctx *c) { return c->dV; }
int oracle_norb(const or_ctx *c, int atom) { return c->sp[c->spc[atom]].norb; }

/* pins: spline value/derivative and orbital values at a displacement */
double oracle_radial(const or_ctx *c, int species, int irad, double r, double *dfdr)
{
    return or_radial(&c->sp[species], irad, r, dfdr);
}

int oracle_phi(const or_ctx *c, int species, const double *d, double *phi, double *grad)
{
    return or_phi(&c->sp[species], d, phi, grad);
}

/* ------------------------------------------------------------------ pair list */
/* All (I, J, n) with |tau_J + n.A - tau_I| < rc_I + rc_J, sorted by (I, J, n1, n2, n3).
 * Writes at most `cap` keys (5 ints each) and returns the total count. */
int64_t oracle_pairs(const or_ctx *c, int64_t cap, int *keys)
{
    int64_t cnt = 0;
    const double *A = c->cell;
    for (int I = 0; I < c->natoms; ++I) {
        for (int J = 0; J < c->natoms; ++J) {
            double rs = c->sp[c->spc[I]].rcut + c->sp[c->spc[J]].rcut;
            double dt[3];
            for (int x = 0; x < 3; ++x) dt[x] = c->tau[3 * J + x] - c->tau[3 * I + x];
            int lo[3], hi[3];
            for (int i = 0; i < 3; ++i) {
                double s = dt[0] * c->g[0 + i] + dt[1] * c->g[3 + i] + dt[2] * c->g[6 + i];
                lo[i] = (int)floor(-s - rs * c->gnorm[i]) - 1;
                hi[i] = (int)ceil(-s + rs * c->gnorm[i]) + 1;
            }
            for (int n1 = lo[0]; n1 <= hi[0]; ++n1)
                for (int n2 = lo[1]; n2 <= hi[1]; ++n2)
                    for (int n3 = lo[2]; n3 <= hi[2]; ++n3) {
                        double v[3];
                        for (int x = 0; x < 3; ++x)
                            v[x] = dt[x] + n1 * A[0 + x] + n2 * A[3 + x] + n3 * A[6 + x];
                        double dist = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                        if (dist < rs) {
                            if (cnt < cap) {
                                int *k = keys + 5 * cnt;
                                k[0] = I; k[1] = J; k[2] = n1; k[3] = n2; k[4] = n3;
                            }
                            ++cnt;
                        }
                    }
        }
    }
    return cnt;
}

/* ------------------------------------------------------------------ block lookup */
static int or_keycmp(const int *a, const int *b)
{
    for (int i = 0; i < 5; ++i) {
        if (a[i] < b[i]) return -1;
        if (a[i] > b[i]) return 1;
    }
    return 0;
}

/* keys must be sorted; returns block index or -1 */
static int64_t or_find(const int *keys, int64_t nblocks, const int *key)
{
    int64_t lo = 0, hi = nblocks - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        int cmp = or_keycmp(keys + 5 * mid, key);
        if (cmp == 0) return mid;
        if (cmp < 0) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* ------------------------------------------------------------------ per-point orbital list */
typedef struct {
    int atom, n[3], norb;
    double d[3];                 /* r - tau_I - R_n */
    double phi[OR_MAXORB];
    double grad[OR_MAXORB * 3];
} or_rec;

static void or_point(const or_ctx *c, int64_t p, double r[3])
{
    int64_t N2 = c->grid[1], N3 = c->grid[2];
    int64_t i = p / (N2 * N3), j = (p / N3) % N2, k = p % N3;
    double s1 = (double)i / c->grid[0], s2 = (double)j / c->grid[1], s3 = (double)k / c->grid[2];
    for (int x = 0; x < 3; ++x) r[x] = s1 * c->cell[0 + x] + s2 * c->cell[3 + x] + s3 * c->cell[6 + x];
}

/* every (atom, image) whose sphere contains r; brute force over all atoms and images */
static int or_collect(const or_ctx *c, const double r[3], or_rec *rec, int cap, int want_grad)
{
    int nrec = 0;
    for (int I = 0; I < c->natoms; ++I) {
        const or_species *S = &c->sp[c->spc[I]];
        const int *lo = c->img_lo + 3 * I, *hi = c->img_hi + 3 * I;
        for (int n1 = lo[0]; n1 <= hi[0]; ++n1)
            for (int n2 = lo[1]; n2 <= hi[1]; ++n2)
                for (int n3 = lo[2]; n3 <= hi[2]; ++n3) {
                    double d[3];
                    for (int x = 0; x < 3; ++x)
                        d[x] = r[x] - (c->tau[3 * I + x] + n1 * c->cell[0 + x] + n2 * c->cell[3 + x] +
                                       n3 * c->cell[6 + x]);
                    double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    if (!(rr < S->rcut)) continue;
                    if (nrec >= cap) return -1;
                    or_rec *q = &rec[nrec++];
                    q->atom = I; q->n[0] = n1; q->n[1] = n2; q->n[2] = n3;
                    q->d[0] = d[0]; q->d[1] = d[1]; q->d[2] = d[2];
                    q->norb = or_phi(S, d, q->phi, want_grad ? q->grad : NULL);
                }
    }
    return nrec;
}

#define OR_MAXREC 512

static int or_nthreads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int or_tid(void)
{
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

int oracle_threads(void) { return or_nthreads(); }

/* H (block store, offsets[b] .. offsets[b]+nI*nJ, row-major) = contribution of the listed
 * grid points (pts == NULL: all points) to V_mu,nu(R) = dV Sum_r phi_mu V phi_nu.  H is
 * overwritten.  Returns 0, or -1 if a point sees more than OR_MAXREC orbital centres, or -2
 * if an overlapping pair is missing from the keys. */
int oracle_vlocal(const or_ctx *c, const double *V, int64_t nblocks, const int *keys,
                  const int64_t *offsets, double *H, int64_t npts, const int64_t *pts)
{
    int64_t nval = offsets[nblocks];
    int nt = or_nthreads();
    double **part = (double **)calloc(nt, sizeof(double *));
    int err = 0;
    memset(H, 0, sizeof(double) * nval);
    int64_t count = pts ? npts : c->npts;
#pragma omp parallel
    {
        int tid = or_tid();
        double *Hp = (double *)calloc(nval, sizeof(double));
        part[tid] = Hp;
        or_rec *rec = (or_rec *)malloc(sizeof(or_rec) * OR_MAXREC);
#pragma omp for schedule(dynamic, 64)
        for (int64_t q = 0; q < count; ++q) {
            int64_t p = pts ? pts[q] : q;
            double r[3];
            or_point(c, p, r);
            int nrec = or_collect(c, r, rec, OR_MAXREC, 0);
            if (nrec < 0) { err = -1; continue; }
            double w = c->dV * V[p];
            for (int x = 0; x < nrec; ++x)
                for (int y = 0; y < nrec; ++y) {
                    int key[5] = {rec[x].atom, rec[y].atom, rec[y].n[0] - rec[x].n[0],
                                  rec[y].n[1] - rec[x].n[1], rec[y].n[2] - rec[x].n[2]};
                    int64_t b = or_find(keys, nblocks, key);
                    if (b < 0) { err = -2; continue; }
                    double *blk = Hp + offsets[b];
                    int nJ = rec[y].norb;
                    for (int mu = 0; mu < rec[x].norb; ++mu) {
                        double a = w * rec[x].phi[mu];
                        for (int nu = 0; nu < nJ; ++nu) blk[mu * nJ + nu] += a * rec[y].phi[nu];
                    }
                }
        }
        free(rec);
    }
    for (int t = 0; t < nt; ++t) {
        if (!part[t]) continue;
        for (int64_t i = 0; i < nval; ++i) H[i] += part[t][i];
        free(part[t]);
    }
    free(part);
    return err;
}

/* rho at the listed points (pts == NULL: all points, rho has npts entries in list order) */
int oracle_rho(const or_ctx *c, int64_t nblocks, const int *keys, const int64_t *offsets,
               const double *DM, double *rho, int64_t npts, const int64_t *pts)
{
    int err = 0;
    int64_t count = pts ? npts : c->npts;
#pragma omp parallel
    {
        or_rec *rec = (or_rec *)malloc(sizeof(or_rec) * OR_MAXREC);
#pragma omp for schedule(dynamic, 64)
        for (int64_t q = 0; q < count; ++q) {
            int64_t p = pts ? pts[q] : q;
            double r[3];
            or_point(c, p, r);
            int nrec = or_collect(c, r, rec, OR_MAXREC, 0);
            if (nrec < 0) { err = -1; rho[q] = 0.0; continue; }
            double acc = 0.0;
            for (int x = 0; x < nrec; ++x)
                for (int y = 0; y < nrec; ++y) {
                    int key[5] = {rec[x].atom, rec[y].atom, rec[y].n[0] - rec[x].n[0],
                                  rec[y].n[1] - rec[x].n[1], rec[y].n[2] - rec[x].n[2]};
                    int64_t b = or_find(keys, nblocks, key);
                    if (b < 0) { err = -2; continue; }
                    const double *blk = DM + offsets[b];
                    int nJ = rec[y].norb;
                    for (int mu = 0; mu < rec[x].norb; ++mu) {
                        double s = 0.0;
                        for (int nu = 0; nu < nJ; ++nu) s += blk[mu * nJ + nu] * rec[y].phi[nu];
                        acc += rec[x].phi[mu] * s;
                    }
                }
            rho[q] = acc;
        }
        free(rec);
    }
    return err;
}

/* dL/dtau (natoms x 3) for L = Sum_blocks Sum DM_mu,nu H_mu,nu, from the listed points:
 *   dL/dtau_K = -dV Sum_r V(r) Sum_{x: atom K} Sum_{mu in x} grad phi_mu .
 *               Sum_{y, nu} (DM(x,y)_mu,nu + DM(y,x)_nu,mu) phi_nu
 * (the basis-motion derivative; the Pulay force is F = -dL/dtau). */
int oracle_dLdtau(const or_ctx *c, const double *V, int64_t nblocks, const int *keys,
                  const int64_t *offsets, const double *DM, double *dL, int64_t npts, const int64_t *pts)
{
    int nt = or_nthreads();
    int err = 0;
    double **part = (double **)calloc(nt, sizeof(double *));
    int64_t count = pts ? npts : c->npts;
#pragma omp parallel
    {
        int tid = or_tid();
        double *Fp = (double *)calloc(3 * (size_t)c->natoms, sizeof(double));
        part[tid] = Fp;
        or_rec *rec = (or_rec *)malloc(sizeof(or_rec) * OR_MAXREC);
#pragma omp for schedule(dynamic, 64)
        for (int64_t q = 0; q < count; ++q) {
            int64_t p = pts ? pts[q] : q;
            double r[3];
            or_point(c, p, r);
            int nrec = or_collect(c, r, rec, OR_MAXREC, 1);
            if (nrec < 0) { err = -1; continue; }
            double w = -c->dV * V[p];
            for (int x = 0; x < nrec; ++x) {
                double g[3] = {0, 0, 0};
                for (int y = 0; y < nrec; ++y) {
                    int key[5] = {rec[x].atom, rec[y].atom, rec[y].n[0] - rec[x].n[0],
                                  rec[y].n[1] - rec[x].n[1], rec[y].n[2] - rec[x].n[2]};
                    int keyT[5] = {rec[y].atom, rec[x].atom, -key[2], -key[3], -key[4]};
                    int64_t b = or_find(keys, nblocks, key);
                    int64_t bt = or_find(keys, nblocks, keyT);
                    if (b < 0 || bt < 0) { err = -2; continue; }
                    const double *blk = DM + offsets[b];
                    const double *blkT = DM + offsets[bt];
                    int nI = rec[x].norb, nJ = rec[y].norb;
                    for (int mu = 0; mu < nI; ++mu) {
                        double s = 0.0;
                        for (int nu = 0; nu < nJ; ++nu)
                            s += (blk[mu * nJ + nu] + blkT[nu * nI + mu]) * rec[y].phi[nu];
                        for (int k = 0; k < 3; ++k) g[k] += rec[x].grad[3 * mu + k] * s;
                    }
                }
                for (int k = 0; k < 3; ++k) Fp[3 * rec[x].atom + k] += w * g[k];
            }
        }
        free(rec);
    }
    memset(dL, 0, sizeof(double) * 3 * c->natoms);
    for (int t = 0; t < nt; ++t) {
        if (!part[t]) continue;
        for (int i = 0; i < 3 * c->natoms; ++i) dL[i] += part[t][i];
        free(part[t]);
    }
    free(part);
    return err;
}

/* Derivative of L with respect to a homogeneous strain eps (stress, Eq. stress: sigma =
 * -(1/Omega) dE/deps).  The strain maps every vector x -> (1 + eps) x: cell, atoms, lattice
 * translations and grid points (the grid keeps its fractional coordinates); the values V(r) on
 * the grid are held fixed and dV scales with det(1 + eps).  With d = r - tau_I - R_n,
 *   dL/deps_ab = delta_ab L
 *              + dV Sum_r V(r) Sum_{x} Sum_{mu in x} d/dx_a phi_mu(d_x) d_x,b .
 *                Sum_{y, nu} (DM(x,y)_mu,nu + DM(y,x)_nu,mu) phi_nu
 * with L = dV Sum_r V(r) rho(r).  out[3 a + b] = dL/deps_ab. */
int oracle_dLdeps(const or_ctx *c, const double *V, int64_t nblocks, const int *keys,
                  const int64_t *offsets, const double *DM, double *out, int64_t npts, const int64_t *pts)
{
    int nt = or_nthreads();
    int err = 0;
    double *part = (double *)calloc((size_t)nt * 10, sizeof(double));
    int64_t count = pts ? npts : c->npts;
#pragma omp parallel
    {
        double *acc = part + 10 * or_tid();   /* [0..8] strain sums, [9] Sum V rho */
        or_rec *rec = (or_rec *)malloc(sizeof(or_rec) * OR_MAXREC);
#pragma omp for schedule(dynamic, 64)
        for (int64_t q = 0; q < count; ++q) {
            int64_t p = pts ? pts[q] : q;
            double r[3];
            or_point(c, p, r);
            int nrec = or_collect(c, r, rec, OR_MAXREC, 1);
            if (nrec < 0) { err = -1; continue; }
            double rho = 0.0;
            for (int x = 0; x < nrec; ++x) {
                double g[3] = {0, 0, 0};
                for (int y = 0; y < nrec; ++y) {
                    int key[5] = {rec[x].atom, rec[y].atom, rec[y].n[0] - rec[x].n[0],
                                  rec[y].n[1] - rec[x].n[1], rec[y].n[2] - rec[x].n[2]};
                    int keyT[5] = {rec[y].atom, rec[x].atom, -key[2], -key[3], -key[4]};
                    int64_t b = or_find(keys, nblocks, key);
                    int64_t bt = or_find(keys, nblocks, keyT);
                    if (b < 0 || bt < 0) { err = -2; continue; }
                    const double *blk = DM + offsets[b];
                    const double *blkT = DM + offsets[bt];
                    int nI = rec[x].norb, nJ = rec[y].norb;
                    for (int mu = 0; mu < nI; ++mu) {
                        double s = 0.0;
                        for (int nu = 0; nu < nJ; ++nu)
                            s += (blk[mu * nJ + nu] + blkT[nu * nI + mu]) * rec[y].phi[nu];
                        for (int k = 0; k < 3; ++k) g[k] += rec[x].grad[3 * mu + k] * s;
                        /* rho(r) = Sum DM phi phi, each ordered pair once (s holds both orders) */
                        rho += 0.5 * rec[x].phi[mu] * s;
                    }
                }
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) acc[3 * a + b] += V[p] * g[a] * rec[x].d[b];
            }
            acc[9] += V[p] * rho;
        }
        free(rec);
    }
    double tot[10] = {0};
    for (int t = 0; t < nt; ++t)
        for (int k = 0; k < 10; ++k) tot[k] += part[10 * t + k];
    free(part);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) out[3 * a + b] = c->dV * tot[3 * a + b] + (a == b ? c->dV * tot[9] : 0.0);
    return err;
}

/* grid points whose distance to some image of atom I is below rc_I (for sampled checks) */
int64_t oracle_points_near_atom(const or_ctx *c, int I, int64_t cap, int64_t *out)
{
    int64_t cnt = 0;
    const or_species *S = &c->sp[c->spc[I]];
    for (int64_t p = 0; p < c->npts; ++p) {
        double r[3];
        or_point(c, p, r);
        int hit = 0;
        const int *lo = c->img_lo + 3 * I, *hi = c->img_hi + 3 * I;
        for (int n1 = lo[0]; n1 <= hi[0] && !hit; ++n1)
            for (int n2 = lo[1]; n2 <= hi[1] && !hit; ++n2)
                for (int n3 = lo[2]; n3 <= hi[2] && !hit; ++n3) {
                    double d[3];
                    for (int x = 0; x < 3; ++x)
                        d[x] = r[x] - (c->tau[3 * I + x] + n1 * c->cell[0 + x] + n2 * c->cell[3 + x] +
                                       n3 * c->cell[6 + x]);
                    if (sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) < S->rcut) hit = 1;
                }
        if (hit) {
            if (cnt < cap) out[cnt] = p;
            ++cnt;
        }
    }
    return cnt;
}

/* ------------------------------------------------------------------ per-block and per-atom forms */
/* Integer grid coordinates (in all space, not wrapped into the cell) of the points within
 * distance rc of centre x: a box in fractional coordinates, per axis. */
static void or_point_box(const or_ctx *c, const double x[3], double rc, int64_t lo[3], int64_t hi[3])
{
    for (int i = 0; i < 3; ++i) {
        double s = x[0] * c->g[0 + i] + x[1] * c->g[3 + i] + x[2] * c->g[6 + i];
        lo[i] = (int64_t)floor((s - rc * c->gnorm[i]) * c->grid[i]) - 1;
        hi[i] = (int64_t)ceil((s + rc * c->gnorm[i]) * c->grid[i]) + 1;
    }
}

static int64_t or_wrap(int64_t i, int64_t n)
{
    int64_t r = i % n;
    return r < 0 ? r + n : r;
}

/* Selected blocks of V_mu,nu(R) written out block by block: for key (I, J, n) with
 * R = n.A, H = dV Sum_r' phi_mu(r' - tau_I) V(r') phi_nu(r' - tau_J - R) over the grid points
 * r' of all space (V periodic), which is the sum over the cell's points and all lattice
 * translations of the definition.  keys[5*b ..] of the nsel requested blocks; out receives the
 * blocks one after another (norb_I x norb_J each, row-major).  Blocks with the same I share one
 * pass over the points of I's sphere (they must be listed consecutively for that to help). */
int oracle_vlocal_blocks(const or_ctx *c, const double *V, int64_t nsel, const int *keys, const int64_t *outoff,
                         double *out)
{
    /* groups of consecutive keys with the same I */
    int64_t ngrp = 0;
    int64_t *g0 = (int64_t *)malloc(sizeof(int64_t) * (nsel + 1));
    for (int64_t b = 0; b < nsel; ++b)
        if (b == 0 || keys[5 * b] != keys[5 * (b - 1)]) g0[ngrp++] = b;
    g0[ngrp] = nsel;
    const double *A = c->cell;
    const int64_t N1 = c->grid[0], N2 = c->grid[1], N3 = c->grid[2];
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t g = 0; g < ngrp; ++g) {
        const int I = keys[5 * g0[g]];
        const or_species *SI = &c->sp[c->spc[I]];
        const double *tI = c->tau + 3 * I;
        int64_t lo[3], hi[3];
        or_point_box(c, tI, SI->rcut, lo, hi);
        double phiI[OR_MAXORB], phiJ[OR_MAXORB];
        for (int64_t b = g0[g]; b < g0[g + 1]; ++b) {
            const or_species *SJ = &c->sp[c->spc[keys[5 * b + 1]]];
            memset(out + outoff[b], 0, sizeof(double) * SI->norb * SJ->norb);
        }
        for (int64_t i = lo[0]; i <= hi[0]; ++i)
            for (int64_t j = lo[1]; j <= hi[1]; ++j)
                for (int64_t k = lo[2]; k <= hi[2]; ++k) {
                    double s1 = (double)i / N1, s2 = (double)j / N2, s3 = (double)k / N3, r[3], dI[3];
                    for (int x = 0; x < 3; ++x) {
                        r[x] = s1 * A[0 + x] + s2 * A[3 + x] + s3 * A[6 + x];
                        dI[x] = r[x] - tI[x];
                    }
                    if (!(sqrt(dI[0] * dI[0] + dI[1] * dI[1] + dI[2] * dI[2]) < SI->rcut)) continue;
                    const double w = c->dV * V[(or_wrap(i, N1) * N2 + or_wrap(j, N2)) * N3 + or_wrap(k, N3)];
                    or_phi(SI, dI, phiI, NULL);
                    for (int64_t b = g0[g]; b < g0[g + 1]; ++b) {
                        const int *key = keys + 5 * b;
                        const or_species *SJ = &c->sp[c->spc[key[1]]];
                        double dJ[3];
                        for (int x = 0; x < 3; ++x)
                            dJ[x] = r[x] - (c->tau[3 * key[1] + x] + key[2] * A[0 + x] + key[3] * A[3 + x] +
                                            key[4] * A[6 + x]);
                        if (!(sqrt(dJ[0] * dJ[0] + dJ[1] * dJ[1] + dJ[2] * dJ[2]) < SJ->rcut)) continue;
                        or_phi(SJ, dJ, phiJ, NULL);
                        double *blk = out + outoff[b];
                        for (int mu = 0; mu < SI->norb; ++mu)
                            for (int nu = 0; nu < SJ->norb; ++nu) blk[mu * SJ->norb + nu] += w * phiI[mu] * phiJ[nu];
                    }
                }
    }
    free(g0);
    return 0;
}

/* dL/dtau_K for selected atoms, written out atom by atom: with L = Sum_blocks Sum DM H,
 *   dL/dtau_K = -dV Sum_r' V(r') Sum_{mu in K} grad phi_mu(r' - tau_K) .
 *               Sum_{blocks (K, J, n)} Sum_{nu in J} (DM(K,J,n)_mu,nu + DM(J,K,-n)_nu,mu) phi_nu(r' - tau_J - n.A)
 * over the grid points r' of all space within rc_K of tau_K (V periodic).  keys/offsets: the
 * full sorted block list and the DM store; out: nsel x 3. */
int oracle_dLdtau_atoms(const or_ctx *c, const double *V, int64_t nblocks, const int *keys, const int64_t *offsets,
                        const double *DM, int64_t nsel, const int *atoms, double *out)
{
    const double *A = c->cell;
    const int64_t N1 = c->grid[0], N2 = c->grid[1], N3 = c->grid[2];
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nsel; ++q) {
        const int K = atoms[q];
        const or_species *SK = &c->sp[c->spc[K]];
        const double *tK = c->tau + 3 * K;
        /* the blocks (K, J, n): a contiguous key range */
        int64_t b0 = 0, b1;
        while (b0 < nblocks && keys[5 * b0] < K) ++b0;
        b1 = b0;
        while (b1 < nblocks && keys[5 * b1] == K) ++b1;
        int64_t *tr = (int64_t *)malloc(sizeof(int64_t) * (b1 - b0 + 1));
        for (int64_t b = b0; b < b1; ++b) {
            const int *k = keys + 5 * b;
            int kt[5] = {k[1], k[0], -k[2], -k[3], -k[4]};
            tr[b - b0] = or_find(keys, nblocks, kt);
            if (tr[b - b0] < 0) err = -2;
        }
        int64_t lo[3], hi[3];
        or_point_box(c, tK, SK->rcut, lo, hi);
        double phiK[OR_MAXORB], gK[OR_MAXORB * 3], phiJ[OR_MAXORB];
        double acc[3] = {0, 0, 0};
        for (int64_t i = lo[0]; i <= hi[0]; ++i)
            for (int64_t j = lo[1]; j <= hi[1]; ++j)
                for (int64_t k = lo[2]; k <= hi[2]; ++k) {
                    double s1 = (double)i / N1, s2 = (double)j / N2, s3 = (double)k / N3, r[3], dK[3];
                    for (int x = 0; x < 3; ++x) {
                        r[x] = s1 * A[0 + x] + s2 * A[3 + x] + s3 * A[6 + x];
                        dK[x] = r[x] - tK[x];
                    }
                    if (!(sqrt(dK[0] * dK[0] + dK[1] * dK[1] + dK[2] * dK[2]) < SK->rcut)) continue;
                    const double w = -c->dV * V[(or_wrap(i, N1) * N2 + or_wrap(j, N2)) * N3 + or_wrap(k, N3)];
                    or_phi(SK, dK, phiK, gK);
                    double g[3] = {0, 0, 0};
                    for (int64_t b = b0; b < b1; ++b) {
                        if (tr[b - b0] < 0) continue;
                        const int *key = keys + 5 * b;
                        const or_species *SJ = &c->sp[c->spc[key[1]]];
                        double dJ[3];
                        for (int x = 0; x < 3; ++x)
                            dJ[x] = r[x] - (c->tau[3 * key[1] + x] + key[2] * A[0 + x] + key[3] * A[3 + x] +
                                            key[4] * A[6 + x]);
                        if (!(sqrt(dJ[0] * dJ[0] + dJ[1] * dJ[1] + dJ[2] * dJ[2]) < SJ->rcut)) continue;
                        or_phi(SJ, dJ, phiJ, NULL);
                        const double *blk = DM + offsets[b], *blkT = DM + offsets[tr[b - b0]];
                        const int nK = SK->norb, nJ = SJ->norb;
                        for (int mu = 0; mu < nK; ++mu) {
                            double s = 0.0;
                            for (int nu = 0; nu < nJ; ++nu) s += (blk[mu * nJ + nu] + blkT[nu * nK + mu]) * phiJ[nu];
                            for (int x = 0; x < 3; ++x) g[x] += gK[3 * mu + x] * s;
                        }
                    }
                    for (int x = 0; x < 3; ++x) acc[x] += w * g[x];
                }
        for (int x = 0; x < 3; ++x) out[3 * q + x] = acc[x];
        free(tr);
    }
    return err;
}
