/*
 * FP64 CPU oracle for the radius-4 acoustic pressure-velocity FDTD step with
 * convolutional PML (CPML) memory variables.
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists so that tests, the smoke check
 * and the CPU-baseline leg of the benchmark can compare the CUDA library with
 * a plain, slow, obviously correct restatement of the method.  It shares no
 * code, header, table or constant with the CUDA library, and the library never
 * calls it.
 *
 * What it computes (paper section 3, "Model"):
 *   - centred derivative, Sec. 3.1:
 *       (delta_d f)_i = (1/h) sum_{l=1..4} a_l (f_{i+l e_d} - f_{i-l e_d})
 *     with the weights a_l passed in (the paper leaves them unprinted; the
 *     Python side derives them);
 *   - leapfrog, Sec. 3.1: velocity half step from p^n, then pressure step
 *     from v^{n+1/2};
 *   - CPML, Sec. 3.2: inside the slab of axis d the derivative delta_d f is
 *     replaced by (1/kappa_d) delta_d f + psi_d with
 *     psi_d <- b_d psi_d + a_d delta_d f   (update with the current derivative,
 *     then use it), for the velocity update (psi_{v,d}) and for the pressure
 *     update (psi_{p,d});
 *   - outside every slab nothing of the CPML is touched (Sec. 3.2: sigma = 0,
 *     kappa = 1, psi = 0 reduce to the interior update).
 * Two options of the same system:
 *   - staggered (the Yee reading of Sec. 3.1): v_d at half nodes i + 1/2,
 *     forward differences p -> v and backward v -> p with the staggered
 *     weights, and the velocity CPML at half-node depths;
 *   - local CPML grading: b_d, a_d per node (bn, an), for a sigma_max taken
 *     from the velocity at the node instead of one reference velocity.
 * Grid values beyond the outermost node are zero (or wrap, in periodic mode,
 * which the energy and dispersion tests use).
 *
 * Layout: every field is a dense [nz][ny][nx] array of doubles, x fastest.
 * Axis numbering: 0 = x, 1 = y, 2 = z.  The CPML coefficient profiles are 1D
 * per axis (length n_axis), one value per node index along that axis.
 *
 * Parity pins live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    long nx, ny, nz;
    double h;                 /* grid spacing, same on every axis */
    double dt;                /* time step */
    double rho;               /* constant density */
    double w[4];              /* derivative weights a_1..a_4 (Sec. 3.1) */
    int periodic;             /* 0: zero values beyond the grid; 1: wrap */
    const double *K;          /* bulk modulus K = rho c^2, [nz][ny][nx] */
    const double *b[3];       /* CPML recursion coefficient b_d per node */
    const double *a[3];       /* CPML recursion coefficient a_d per node */
    const double *kinv[3];    /* 1/kappa_d per node */
    const unsigned char *slab[3]; /* 1 where the node lies in a d-slab */
    const double *rho_n;      /* density per node [nz][ny][nx], or NULL: rho everywhere */
    double kr[3];             /* elliptic anisotropy: modulus along axis d = kr[d] K (1 = isotropic) */
    int staggered;            /* 1: v_d at half nodes i + 1/2 along d (the Yee reading of Sec. 3.1) */
    const double *bv[3];      /* staggered: CPML coefficients of the velocity nodes (half-node depth) */
    const double *av[3];
    const double *kinvv[3];
    const double *bn[3];      /* local grading: b_d per node [nz][ny][nx] (NULL: the 1D b[d]) */
    const double *an[3];      /* local grading: a_d per node (NULL: the 1D a[d]) */
    /* 16-bit storage form: the arithmetic stays FP64, and every stored field
     * is rounded to nearest (ties to even) in the storage format when it is
     * written back: store_bits = 11 (FP16: 11-bit significand, normal
     * exponents >= -14, largest finite 65504) or 8 (BF16: 8-bit significand,
     * normal exponents >= -126); 0 = no rounding.  Fields are scaled before
     * rounding as the form stores them: p and psi_v by scale_p, v and psi_p by
     * scale_p * scale_v.  store_mask selects the fields rounded (bit 0 p,
     * 1 v, 2 psi_v, 3 psi_p). */
    int store_bits;
    int store_mask;
    double scale_p, scale_v;
} og_grid;

/* x rounded to the nearest value with a `bits`-bit significand whose
 * exponent is at least emin (below it the quantum stays 2^(emin - bits + 1),
 * the subnormal range), ties to even; beyond `fmax` the result is +-inf. */
static double og_round_fmt(double x, int bits, int emin, double fmax)
{
    if (x == 0.0 || x != x)
        return x;
    int e;
    frexp(x, &e);               /* |x| = m 2^e, m in [0.5, 1): exponent of the leading bit is e - 1 */
    int lead = e - 1;
    if (lead < emin)
        lead = emin;
    const double q = ldexp(1.0, lead - (bits - 1));
    const double r = nearbyint(x / q) * q;   /* default rounding mode: to nearest, ties to even */
    if (fabs(r) > fmax)
        return x > 0 ? HUGE_VAL : -HUGE_VAL;
    return r;
}

/* og_round_fmt for the two storage formats (bits = 11: FP16, 8: BF16); for tests. */
double og_round16(double x, int bits)
{
    return bits == 11 ? og_round_fmt(x, 11, -14, 65504.0) : og_round_fmt(x, 8, -126, 3.3895313892515355e38);
}

/* A stored value of field class `cls` (bit of store_mask) in physical units. */
static double og_store(const og_grid *g, int cls, double x)
{
    if (!g->store_bits || !(g->store_mask & (1 << cls)))
        return x;
    const double s = (cls == 0 || cls == 2) ? g->scale_p : g->scale_p * g->scale_v;
    const double y = g->store_bits == 11 ? og_round_fmt(x * s, 11, -14, 65504.0)
                                         : og_round_fmt(x * s, 8, -126, 3.3895313892515355e38);
    return y / s;
}

/* CPML coefficients of axis d at node i (axis index k) */
static double og_b(const og_grid *g, int d, long i, long k)
{
    return g->bn[d] ? g->bn[d][i] : g->b[d][k];
}

static double og_a(const og_grid *g, int d, long i, long k)
{
    return g->an[d] ? g->an[d][i] : g->a[d][k];
}

/* density at node i (collocated with p and v, Sec. 3.1) */
static double og_rho(const og_grid *g, long i)
{
    return g->rho_n ? g->rho_n[i] : g->rho;
}

typedef struct {
    double *p;
    double *v[3];
    double *psiv[3];          /* psi_{v,d}: memory of delta_d p */
    double *psip[3];          /* psi_{p,d}: memory of delta_d v_d */
} og_state;

/* f at (z, y, x); zero outside the grid unless periodic. */
static double og_at(const og_grid *g, const double *f, long z, long y, long x)
{
    if (g->periodic) {
        x = ((x % g->nx) + g->nx) % g->nx;
        y = ((y % g->ny) + g->ny) % g->ny;
        z = ((z % g->nz) + g->nz) % g->nz;
    } else if (x < 0 || x >= g->nx || y < 0 || y >= g->ny || z < 0 || z >= g->nz) {
        return 0.0;
    }
    return f[(z * g->ny + y) * g->nx + x];
}

/* Centred radius-4 derivative of f along `axis` at (z, y, x), Sec. 3.1. */
static double og_deriv(const og_grid *g, const double *f, int axis, long z, long y, long x)
{
    long dz = axis == 2, dy = axis == 1, dx = axis == 0;
    double s = 0.0;
    for (int l = 1; l <= 4; l++) {
        double fp = og_at(g, f, z + l * dz, y + l * dy, x + l * dx);
        double fm = og_at(g, f, z - l * dz, y - l * dy, x - l * dx);
        s += g->w[l - 1] * (fp - fm);
    }
    return s / g->h;
}

/* Staggered derivatives (radius 4, weights w = c_1..c_4 for the offsets
 * 1/2, 3/2, 5/2, 7/2).  v_d[i] lives at i + 1/2 along d:
 *   forward  (p -> v):  (1/h) sum_l c_l (f_{i+l} - f_{i+1-l})   at i + 1/2,
 *   backward (v -> p):  (1/h) sum_l c_l (f_{i+l-1} - f_{i-l})   at i.
 * With zero values beyond the grid the backward operator is minus the
 * transpose of the forward one. */
static double og_deriv_fwd(const og_grid *g, const double *f, int axis, long z, long y, long x)
{
    long dz = axis == 2, dy = axis == 1, dx = axis == 0;
    double s = 0.0;
    for (int l = 1; l <= 4; l++) {
        double fp = og_at(g, f, z + l * dz, y + l * dy, x + l * dx);
        double fm = og_at(g, f, z + (1 - l) * dz, y + (1 - l) * dy, x + (1 - l) * dx);
        s += g->w[l - 1] * (fp - fm);
    }
    return s / g->h;
}

static double og_deriv_bwd(const og_grid *g, const double *f, int axis, long z, long y, long x)
{
    long dz = axis == 2, dy = axis == 1, dx = axis == 0;
    double s = 0.0;
    for (int l = 1; l <= 4; l++) {
        double fp = og_at(g, f, z + (l - 1) * dz, y + (l - 1) * dy, x + (l - 1) * dx);
        double fm = og_at(g, f, z - l * dz, y - l * dy, x - l * dx);
        s += g->w[l - 1] * (fp - fm);
    }
    return s / g->h;
}

static long og_axis_index(int axis, long z, long y, long x)
{
    return axis == 0 ? x : (axis == 1 ? y : z);
}

/* Velocity half step: v_d <- v_d - (dt/rho) [ (1/kappa_d) delta_d p + psi_{v,d} ]
 * (interior: v_d <- v_d - (dt/rho) delta_d p).  Reads only p, so the update of
 * v in place is a Jacobi update. */
void og_velocity_stage(const og_grid *g, og_state *st)
{
    long nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for schedule(static)
    for (long z = 0; z < nz; z++)
        for (long y = 0; y < ny; y++)
            for (long x = 0; x < nx; x++) {
                long i = (z * ny + y) * nx + x;
                for (int d = 0; d < 3; d++) {
                    double gd = g->staggered ? og_deriv_fwd(g, st->p, d, z, y, x) : og_deriv(g, st->p, d, z, y, x);
                    long k = og_axis_index(d, z, y, x);
                    if (g->slab[d][k]) {
                        const double *kinv = g->staggered ? g->kinvv[d] : g->kinv[d];
                        const double b = g->staggered ? g->bv[d][k] : og_b(g, d, i, k);
                        const double a = g->staggered ? g->av[d][k] : og_a(g, d, i, k);
                        st->psiv[d][i] = b * st->psiv[d][i] + a * gd;
                        gd = kinv[k] * gd + st->psiv[d][i];
                        st->psiv[d][i] = og_store(g, 2, st->psiv[d][i]);
                    }
                    st->v[d][i] -= g->dt / og_rho(g, i) * gd;
                }
            }
}

/* Pressure step: p <- p - dt K sum_d [ (1/kappa_d) delta_d v_d + psi_{p,d} ].
 * Reads only v, so the update of p in place is a Jacobi update.  If s_out is
 * not NULL it receives the bracket sum_d[...] per node (used by the adjoint to
 * form dJ/dK). */
void og_pressure_stage(const og_grid *g, og_state *st, double *s_out)
{
    long nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for schedule(static)
    for (long z = 0; z < nz; z++)
        for (long y = 0; y < ny; y++)
            for (long x = 0; x < nx; x++) {
                long i = (z * ny + y) * nx + x;
                double s = 0.0;
                for (int d = 0; d < 3; d++) {
                    double hd = g->staggered ? og_deriv_bwd(g, st->v[d], d, z, y, x)
                                             : og_deriv(g, st->v[d], d, z, y, x);
                    long k = og_axis_index(d, z, y, x);
                    if (g->slab[d][k]) {
                        st->psip[d][i] = og_b(g, d, i, k) * st->psip[d][i] + og_a(g, d, i, k) * hd;
                        hd = g->kinv[d][k] * hd + st->psip[d][i];
                        st->psip[d][i] = og_store(g, 3, st->psip[d][i]);
                    }
                    s += g->kr[d] * hd;
                }
                st->p[i] -= g->dt * g->K[i] * s;
                if (s_out)
                    s_out[i] = s;
            }
}

/*
 * 16-bit storage form: p and v are written back rounded once the step's
 * pressure update and source are done (the pressure update itself uses the
 * unrounded new velocities, which a fused step keeps in registers).
 */
void og_store_state(const og_grid *g, og_state *st)
{
    long n = g->nx * g->ny * g->nz;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        st->p[i] = og_store(g, 0, st->p[i]);
        for (int d = 0; d < 3; d++)
            st->v[d][i] = og_store(g, 1, st->v[d][i]);
    }
}

/*
 * Run `nsteps` full steps starting at time index n0.  After the pressure
 * update of step n the source wavelet sample w[n] is added at `src`
 * (additive pressure source, amplitude as given), then every receiver samples
 * p: traces[(n - n0) * nrec + r] = p[rec_r].  src[0] < 0 disables the source;
 * wavelet samples beyond nt_w count as zero.  rec holds (z, y, x) triples.
 */
void og_run(const og_grid *g, og_state *st, long n0, long nsteps,
            const long *src, const double *wavelet, long nt_w,
            long nrec, const long *rec, double *traces)
{
    for (long s = 0; s < nsteps; s++) {
        long n = n0 + s;
        og_velocity_stage(g, st);
        og_pressure_stage(g, st, NULL);
        if (src && src[0] >= 0 && wavelet && n < nt_w)
            st->p[(src[0] * g->ny + src[1]) * g->nx + src[2]] += wavelet[n];
        if (g->store_bits)
            og_store_state(g, st);
        for (long r = 0; r < nrec; r++) {
            long z = rec[3 * r], y = rec[3 * r + 1], x = rec[3 * r + 2];
            traces[s * nrec + r] = st->p[(z * g->ny + y) * g->nx + x];
        }
    }
}

/*
 * (D_d^T y) accumulated into out, written as the literal transpose of the
 * gather in og_deriv: every node i sends +a_l/h * y_i to i + l e_d and
 * -a_l/h * y_i to i - l e_d (targets outside the grid receive nothing, since
 * the gather never reads there; periodic mode wraps).  Serial on purpose.
 */
/*
 * Transposes of the staggered derivatives, as scatters of the gathers in
 * og_deriv_fwd / og_deriv_bwd: node i sends +c_l/h y_i to i + l (fwd) or
 * i + l - 1 (bwd) and -c_l/h y_i to i + 1 - l (fwd) or i - l (bwd); targets
 * outside the grid receive nothing (periodic mode wraps).
 */
static void og_stag_transpose_acc(const og_grid *g, const double *y, int axis, int fwd, double *out)
{
    long nx = g->nx, ny = g->ny, nz = g->nz;
    long dz = axis == 2, dy = axis == 1, dx = axis == 0;
    for (long z = 0; z < nz; z++)
        for (long yy = 0; yy < ny; yy++)
            for (long x = 0; x < nx; x++) {
                double val = y[(z * ny + yy) * nx + x] / g->h;
                if (val == 0.0)
                    continue;
                for (int l = 1; l <= 4; l++) {
                    const long offs[2] = {fwd ? l : l - 1, fwd ? 1 - l : -l};
                    for (int s = 0; s < 2; s++) {
                        long tz = z + offs[s] * dz, ty = yy + offs[s] * dy, tx = x + offs[s] * dx;
                        if (g->periodic) {
                            tx = ((tx % nx) + nx) % nx;
                            ty = ((ty % ny) + ny) % ny;
                            tz = ((tz % nz) + nz) % nz;
                        } else if (tx < 0 || tx >= nx || ty < 0 || ty >= ny || tz < 0 || tz >= nz) {
                            continue;
                        }
                        out[(tz * ny + ty) * nx + tx] += (s == 0 ? 1.0 : -1.0) * g->w[l - 1] * val;
                    }
                }
            }
}

static void og_deriv_transpose_acc(const og_grid *g, const double *y, int axis, double *out)
{
    long nx = g->nx, ny = g->ny, nz = g->nz;
    long dz = axis == 2, dy = axis == 1, dx = axis == 0;
    for (long z = 0; z < nz; z++)
        for (long yy = 0; yy < ny; yy++)
            for (long x = 0; x < nx; x++) {
                double val = y[(z * ny + yy) * nx + x] / g->h;
                if (val == 0.0)
                    continue;
                for (int l = 1; l <= 4; l++) {
                    for (int sgn = -1; sgn <= 1; sgn += 2) {
                        long tz = z + sgn * l * dz, ty = yy + sgn * l * dy, tx = x + sgn * l * dx;
                        if (g->periodic) {
                            tx = ((tx % nx) + nx) % nx;
                            ty = ((ty % ny) + ny) % ny;
                            tz = ((tz % nz) + nz) % nz;
                        } else if (tx < 0 || tx >= nx || ty < 0 || ty >= ny || tz < 0 || tz >= nz) {
                            continue;
                        }
                        out[(tz * ny + ty) * nx + tx] += sgn * g->w[l - 1] * val;
                    }
                }
            }
}

/*
 * Adjoint (transpose) of one full step n, for the misfit gradient.
 *
 * fwd   : forward state at the START of step n (p^n, v^{n-1/2}, psi before the
 *         step); not modified.
 * adj   : on entry, the adjoint of the state at the END of step n (after the
 *         caller has added the receiver residuals of step n to adj->p); on
 *         exit, the adjoint of the state at the start of step n.
 * gradK : accumulates dJ/dK per node (may be NULL).
 * gprof : accumulates dJ/d(b_d, a_d, kinv_d) per axis and node index, layout
 *         [axis][coef][nmax] with coef 0 = b, 1 = a, 2 = kinv (may be NULL).
 *
 * The forward step, written as a sequence of assignments
 *   g_d  = D_d p ;  psiv_d' = b psiv_d + a g_d ;  v_d' = v_d - dt/rho (kinv g_d + psiv_d')
 *   h_d  = D_d v_d' ; psip_d' = b psip_d + a h_d ;
 *   p' = p - dt K sum_d kr_d (kinv h_d + psip_d')
 * (CPML terms only inside the d-slab; kr_d = 1 unless anisotropic), is
 * transposed assignment by assignment in reverse order.  The source term is a
 * constant and has no adjoint.
 * The staggered form transposes its own operators (D+ for p -> v, D- for
 * v -> p) and the half-node velocity profiles; with the local grading (bn,
 * an) the per-node coefficients are transposed the same way.  gprof, per
 * axis and node index of the node profiles, is for the collocated form with
 * 1D profiles only.
 */
void og_adjoint_step(const og_grid *g, const og_state *fwd, og_state *adj,
                     double *gradK, double *gprof, long nmax)
{
    long nx = g->nx, ny = g->ny, nz = g->nz, nn = nx * ny * nz;
    size_t bytes = (size_t)nn * sizeof(double);

    /* --- recompute the forward quantities of step n --- */
    og_state f;
    double *buf = calloc((size_t)11 * nn, sizeof(double));
    f.p = buf;
    for (int d = 0; d < 3; d++) {
        f.v[d] = buf + (1 + d) * nn;
        f.psiv[d] = buf + (4 + d) * nn;
        f.psip[d] = buf + (7 + d) * nn;
    }
    double *s_all = buf + 10 * nn;     /* bracket of the pressure update */
    memcpy(f.p, fwd->p, bytes);
    for (int d = 0; d < 3; d++) {
        memcpy(f.v[d], fwd->v[d], bytes);
        memcpy(f.psiv[d], fwd->psiv[d], bytes);
        memcpy(f.psip[d], fwd->psip[d], bytes);
    }
    double *g_d[3], *h_d[3];
    for (int d = 0; d < 3; d++) {
        g_d[d] = malloc(bytes);
        h_d[d] = malloc(bytes);
    }
    for (long z = 0; z < nz; z++)
        for (long y = 0; y < ny; y++)
            for (long x = 0; x < nx; x++)
                for (int d = 0; d < 3; d++)
                    g_d[d][(z * ny + y) * nx + x] = g->staggered ? og_deriv_fwd(g, f.p, d, z, y, x)
                                                                 : og_deriv(g, f.p, d, z, y, x);
    og_velocity_stage(g, &f);          /* f.v = v^{n+1/2}, f.psiv = psiv after */
    for (long z = 0; z < nz; z++)
        for (long y = 0; y < ny; y++)
            for (long x = 0; x < nx; x++)
                for (int d = 0; d < 3; d++)
                    h_d[d][(z * ny + y) * nx + x] = g->staggered ? og_deriv_bwd(g, f.v[d], d, z, y, x)
                                                                 : og_deriv(g, f.v[d], d, z, y, x);
    og_pressure_stage(g, &f, s_all);   /* s_all = bracket of the pressure update */

    /* --- p' = p - dt K sum_d (kinv h_d + psip_d') ;  psip_d' = b psip_d + a h_d --- */
    double *lam_h[3], *lam_g[3];
    for (int d = 0; d < 3; d++) {
        lam_h[d] = calloc((size_t)nn, sizeof(double));
        lam_g[d] = calloc((size_t)nn, sizeof(double));
    }
    for (long z = 0; z < nz; z++)
        for (long y = 0; y < ny; y++)
            for (long x = 0; x < nx; x++) {
                long i = (z * ny + y) * nx + x;
                double lp = adj->p[i];
                if (gradK)
                    gradK[i] += -g->dt * s_all[i] * lp;
                double q0 = -g->dt * g->K[i] * lp;   /* adjoint of the bracket sum */
                for (int d = 0; d < 3; d++) {
                    long k = og_axis_index(d, z, y, x);
                    double q = g->kr[d] * q0;         /* adjoint of axis d's bracket */
                    if (g->slab[d][k]) {
                        double lpsi = adj->psip[d][i] + q;   /* total adjoint of psip_d' */
                        lam_h[d][i] = g->kinv[d][k] * q + og_a(g, d, i, k) * lpsi;
                        if (gprof) {
                            gprof[(d * 3 + 0) * nmax + k] += lpsi * fwd->psip[d][i];
                            gprof[(d * 3 + 1) * nmax + k] += lpsi * h_d[d][i];
                            gprof[(d * 3 + 2) * nmax + k] += q * h_d[d][i];
                        }
                        adj->psip[d][i] = og_b(g, d, i, k) * lpsi;
                    } else {
                        lam_h[d][i] = q;
                    }
                }
                /* identity part of p' = p - ...: adj->p keeps its value */
            }
    /* h_d = D_d v_d'  =>  lam(v_d') += D_d^T lam_h_d  (D- in the staggered form) */
    for (int d = 0; d < 3; d++) {
        if (g->staggered)
            og_stag_transpose_acc(g, lam_h[d], d, 0, adj->v[d]);
        else
            og_deriv_transpose_acc(g, lam_h[d], d, adj->v[d]);
    }

    /* --- v_d' = v_d - dt/rho (kinv g_d + psiv_d') ; psiv_d' = b psiv_d + a g_d --- */
    for (long z = 0; z < nz; z++)
        for (long y = 0; y < ny; y++)
            for (long x = 0; x < nx; x++) {
                long i = (z * ny + y) * nx + x;
                for (int d = 0; d < 3; d++) {
                    long k = og_axis_index(d, z, y, x);
                    double r = -g->dt / og_rho(g, i) * adj->v[d][i];
                    if (g->slab[d][k]) {
                        /* velocity coefficients: half-node profiles in the staggered form */
                        const double bvk = g->staggered ? g->bv[d][k] : og_b(g, d, i, k);
                        const double avk = g->staggered ? g->av[d][k] : og_a(g, d, i, k);
                        const double kvk = g->staggered ? g->kinvv[d][k] : g->kinv[d][k];
                        double lpsi = adj->psiv[d][i] + r;
                        lam_g[d][i] = kvk * r + avk * lpsi;
                        if (gprof) {
                            gprof[(d * 3 + 0) * nmax + k] += lpsi * fwd->psiv[d][i];
                            gprof[(d * 3 + 1) * nmax + k] += lpsi * g_d[d][i];
                            gprof[(d * 3 + 2) * nmax + k] += r * g_d[d][i];
                        }
                        adj->psiv[d][i] = bvk * lpsi;
                    } else {
                        lam_g[d][i] = r;
                    }
                    /* identity part of v_d' = v_d - ...: adj->v keeps its value */
                }
            }
    /* g_d = D_d p  =>  lam(p) += sum_d D_d^T lam_g_d  (D+ in the staggered form) */
    for (int d = 0; d < 3; d++) {
        if (g->staggered)
            og_stag_transpose_acc(g, lam_g[d], d, 1, adj->p);
        else
            og_deriv_transpose_acc(g, lam_g[d], d, adj->p);
    }

    for (int d = 0; d < 3; d++) {
        free(lam_h[d]);
        free(lam_g[d]);
        free(g_d[d]);
        free(h_d[d]);
    }
    free(buf);
}

/* Layout version of og_grid/og_state; the Python side checks it on load. */
long og_version(void) { return 2; }

/* Threads an OpenMP loop of this library uses (1 when built without OpenMP);
 * reported next to timings of the oracle. */
#ifdef _OPENMP
#include <omp.h>
long og_threads(void) { return omp_get_max_threads(); }
#else
long og_threads(void) { return 1; }
#endif
