/*
 * lym1_oracle.c -- plain, slow FP64 reference ("oracle") for one substep of the
 * Lydion M1 method for Lyman-alpha transfer on a 2D Cartesian grid or an
 * axisymmetric (R, Z) grid (arXiv 2606.02711).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline arm may load this file's library.  The GPU product
 * path does not link, import or call it, and this file shares no code with the
 * GPU path (its own constants, its own exp/expm1, its own Dawson function).
 *
 * What it computes, in the paper's order (Sec. 2.1, "overall update scheme"):
 *   A0  frequency grid (Sec. 2.1, grid paragraph), bin-averaged Voigt profile
 *       <H>_k (App. A, bin-averaged Voigt eq. and the I(x,a) integral),
 *       emission fractions from phi_nu = H/sqrt(pi) (Sec. 2.1 step 2).
 *   A1  linear reconstruction of J and f = H/J with MinMod; |f| > 1 rescaled
 *       (Sec. 2.1 step 1 and its footnote); M1 closure (Levermore closure eq.).
 *   A2  asymptotic-preserving GLF flux for J (corrected GLF flux eq.), the
 *       interpolation factor eps and face optical depth (Sec. 2.1 step 1),
 *       the modified GLF flux for K, upwind advection of uJ/c and uH/c.
 *   A3  explicit forward-Euler update including the -grad(u):K/c work term.
 *   A4  implicit emission/absorption/destruction (absorption step eqs.).
 *   A5  radiation force from the change of H in A4 (Sec. 2.3 force eq.).
 *   A6  implicit (BDF1) frequency diffusion + recoil + Doppler solve per cell
 *       with the exponential scheme (App. A), then H = (J_new/J_old) H.
 *   A7  energy bookkeeping with compensated (Neumaier) sums.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - Cartesian geometry: face optical depth tau = aF_i dx/2 + aF_{i+1} dx/2,
 *     D:grad u = Dxx dux/dx + Dyy duy/dy + Dxy (dux/dy + duy/dx).
 *   - outflow boundaries: two ghost layers per side, either copying the edge
 *     cell (zero gradient, the default) or, for a cloud surrounded by vacuum
 *     (Sec. 4 test set-ups), holding no radiation while the opacities and
 *     velocities are copied, so that radiation leaves but never enters.  The
 *     zero-gradient ghosts let an inward flux at the edge feed the edge cell,
 *     which grew without bound in the vacuum gap of the 256^2 cone test.
 *   - face velocity = mean of the two cells; the upwind donor is the
 *     reconstructed state on the upwind side.
 *   - velocity gradients by central differences over the two neighbours.
 *   - the K-flux dissipation term uses the jump of the same H component.
 *   - the diffusion part of the J flux is (1-eps)(J_{i+1}-J_i)/(3 tau), and 0
 *     where tau = 0 (then eps = 1).
 *   - A6: the exponential-scheme leakage coefficients are evaluated with a
 *     common exponential factor taken out so that nothing overflows at large
 *     Peclet numbers, and the tridiagonal system is eliminated in its
 *     conservative (flux) form carrying the diagonal-dominance margin, which
 *     keeps every step free of subtraction.  Both are exact rearrangements of
 *     the App. A equations.
 *   - phi and chi are evaluated with this file's own exp/expm1 (Cody-Waite
 *     argument reduction + Taylor polynomial), not lookup tables.
 *   - no FMA contraction: build with -ffp-contract=off.
 *   - a per-cell gas temperature (App. A evaluates <H>_k, the Doppler width and a_v
 *     at each cell): A0 runs once per cell at its own T with the same routine
 *     as for a uniform T; alpha = n_HI sigma0(T), the recoil factor h/(k_B T)
 *     and the step-3 prefactor dnu_D^2/2 are per cell.
 *   - axisymmetric (R, Z) geometry (the paper's test and RHD set-ups, Sec. 4):
 *     finite volumes per radian with R faces of area R dZ and Z faces of area
 *     (R+^2 - R-^2)/2; the R component of div K carries the hoop source
 *     K_phiphi <1/R> with <1/R> = dR dZ / Vol, which makes a uniform isotropic
 *     field exactly steady; the work term and step 3's D:grad u add
 *     D_phiphi <u_R/R>, with <u_R/R> from the two R-face velocities; the face
 *     optical depth uses the centroid-to-face distances (Sec. 2.1 step 1);
 *     the axis and the midplane are mirrors (H_R, u_R flip across the axis,
 *     H_Z, u_Z across the midplane), the outer edges outflow; MinMod slopes
 *     use cell indices (uniform geometric centres); the cell luminosity is
 *     emitted into the full ring volume 2 pi Vol.
 *
 * Parity pins (tests/test_oracle_*.py): printed N_nu = 194, sigma0 and a_v
 * scalings, Dawson vs scipy, <H> vs quadrature, closure and eps limits,
 * conservation of energy to round-off, realisability, free-streaming beam,
 * Gaussian diffusion closed form, thin-slab force multiplier, step-3 vs dense
 * and exact-rational solves, recoil-only equilibrium, central-difference
 * limit vs a banded solver; in (R, Z): the thin-sphere force multiplier
 * tau eta / 4, a steady uniform isotropic field, the Hubble-flow work term;
 * under a temperature field: a uniform field equals the scalar T bit for bit,
 * and cells at two temperatures equal one-cell runs at their own T.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- physical constants, cgs (CODATA 2018) ---- */
#define O_PI 3.14159265358979323846
#define O_SQRTPI 1.772453850905516
#define O_C 2.99792458e10          /* speed of light, cm/s */
#define O_HPL 6.62607015e-27       /* Planck constant, erg s */
#define O_KB 1.380649e-16          /* Boltzmann constant, erg/K */
#define O_ME 9.1093837015e-28      /* electron mass, g */
#define O_QE 4.803204712570263e-10 /* elementary charge, esu */
#define O_MH 1.67353284e-24        /* hydrogen atom mass, g */
#define O_NU_LYA (O_C / 1215.67e-8) /* Lya line-centre frequency, Hz */
#define O_NU_LYC 3.28805e15        /* H ionisation threshold frequency, Hz */
#define O_A_LYA 6.265e8            /* Lya Einstein A, 1/s */
#define O_F12 0.4162               /* Lya oscillator strength */

/* ======================================================================
 * Own exp / expm1: Cody-Waite argument reduction x = n ln2 + r, |r| <= ln2/2,
 * then a degree-13 Taylor polynomial for expm1(r) (remainder < 1.2e-17 |r|).
 * ln2 is split into a 32-significant-bit head (so n*LN2_HI is exact for
 * |n| < 2^20) and the rounded tail.
 * ====================================================================== */
static const double O_LN2_HI = 0x1.62e42feep-1;
static const double O_LN2_LO = 0x1.a39ef35793c76p-33;
static const double O_INV_LN2 = 0x1.71547652b82fep+0;

static double o_pow2i(int n) /* exact 2^n for -1022 <= n <= 1023 */
{
    uint64_t b = (uint64_t)(n + 1023) << 52;
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
}

static double o_expm1_poly(double r)
{
    double q = 1.0 / 6227020800.0; /* 1/13! */
    q = q * r + 1.0 / 479001600.0; /* 1/12! */
    q = q * r + 1.0 / 39916800.0;  /* 1/11! */
    q = q * r + 1.0 / 3628800.0;   /* 1/10! */
    q = q * r + 1.0 / 362880.0;    /* 1/9! */
    q = q * r + 1.0 / 40320.0;     /* 1/8! */
    q = q * r + 1.0 / 5040.0;      /* 1/7! */
    q = q * r + 1.0 / 720.0;       /* 1/6! */
    q = q * r + 1.0 / 120.0;       /* 1/5! */
    q = q * r + 1.0 / 24.0;        /* 1/4! */
    q = q * r + 1.0 / 6.0;         /* 1/3! */
    q = q * r + 1.0 / 2.0;         /* 1/2! */
    return r + (r * r) * q;
}

static void o_reduce(double x, int *n, double *r)
{
    double t = floor(x * O_INV_LN2 + 0.5);
    *n = (int)t;
    *r = (x - t * O_LN2_HI) - t * O_LN2_LO;
}

double lym1o_exp(double x)
{
    if (x != x) return x;
    if (x > 709.782712893384) return INFINITY;
    if (x < -745.2) return 0.0;
    int n;
    double r;
    o_reduce(x, &n, &r);
    double s = 1.0 + o_expm1_poly(r);
    if (n > 1023) return (s * 2.0) * o_pow2i(n - 1);
    if (n >= -1022) return s * o_pow2i(n);
    return (s * o_pow2i(n + 1022)) * o_pow2i(-1022);
}

double lym1o_expm1(double x)
{
    if (x != x) return x;
    if (x > 709.782712893384) return INFINITY;
    if (x < -745.2) return -1.0;
    int n;
    double r;
    o_reduce(x, &n, &r);
    double p = o_expm1_poly(r);
    if (n == 0) return p;
    if (n < -1022) return -1.0;
    if (n > 1023) return (p + 1.0) * 2.0 * o_pow2i(n - 1);
    double t = o_pow2i(n);
    return t * p + (t - 1.0);
}

/* ======================================================================
 * Dawson's integral F(x) = exp(-x^2) int_0^x exp(y^2) dy, needed by the
 * bin-averaged Voigt profile (App. A, I(x,a) integral).
 *   |x| < 0.2 : Maclaurin series  F = sum_n (-2)^n x^(2n+1) / (2n+1)!!
 *   |x| < 10  : Rybicki (1989) sampling-theorem sum
 *               F(x) ~ pi^(-1/2) sum_{n odd} exp(-(x - n h)^2) / n, h = 0.2,
 *               whose error is of order exp(-(pi/2h)^2) ~ 1e-27
 *   |x| >= 10 : asymptotic series F ~ (1/2x) sum_n (2n-1)!! / (2x^2)^n
 * ====================================================================== */
double lym1o_dawson(double x)
{
    double ax = fabs(x), f;
    if (ax < 0.2) {
        double x2 = ax * ax, term = ax;
        f = ax;
        for (int n = 1; n <= 12; ++n) {
            term = (term * (-2.0 * x2)) / (2.0 * n + 1.0);
            f += term;
        }
    } else if (ax < 10.0) {
        const double h = 0.2;
        int n_lo = (int)ceil((ax - 8.0) / h), n_hi = (int)floor((ax + 8.0) / h);
        double s = 0.0;
        for (int n = n_lo; n <= n_hi; ++n) {
            if ((n & 1) == 0) continue;
            double d = ax - n * h;
            s += exp(-d * d) / n;
        }
        f = s / O_SQRTPI;
    } else {
        double y = 1.0 / (2.0 * ax * ax), term = 1.0, s = 1.0;
        for (int n = 1; n <= 20; ++n) {
            term = term * ((2.0 * n - 1.0) * y);
            s += term;
        }
        f = s / (2.0 * ax);
    }
    return (x < 0.0) ? -f : f;
}

/* ---- line constants at temperature T (Sec. 2.1 grid paragraph) ---- */
void lym1o_line(double T, double *out3 /* dnuD, a_v, sigma0 */)
{
    double dnuD = (O_NU_LYA * sqrt((2.0 * O_KB * T) / O_MH)) / O_C;
    out3[0] = dnuD;
    out3[1] = O_A_LYA / ((4.0 * O_PI) * dnuD);
    out3[2] = ((O_SQRTPI * (O_QE * O_QE)) * O_F12) / ((O_ME * O_C) * dnuD);
}

/*
 * Frequency grid (Sec. 2.1, grid paragraph): symmetric in dnu = nu - nu_Lya,
 * the two central bins of width dnu_D(T_min), widths growing by q outwards,
 * |dnu| <= min(1e5 dnu_D(T_min), 0.99 nu_Lya, nu_LyC - nu_Lya).  The last bin on
 * each side is the one that crosses the limit, truncated at it.  Writes the
 * 2M+1 ascending edges and returns N = 2M (or -1 if max_edges is too small).
 */
int lym1o_freq_grid(double T_min, double q, double *edges, int max_edges)
{
    double ln[3];
    lym1o_line(T_min, ln);
    double w0 = ln[0];
    double lim = 1e5 * w0;
    if (0.99 * O_NU_LYA < lim) lim = 0.99 * O_NU_LYA;
    if (O_NU_LYC - O_NU_LYA < lim) lim = O_NU_LYC - O_NU_LYA;
    /* positive-side edges e_0 = 0 < e_1 < ... < e_M = lim */
    double *pos = (double *)malloc(100000 * sizeof(double));
    int M = 0;
    double e = 0.0, w = w0;
    pos[0] = 0.0;
    while (1) {
        double next = e + w;
        M += 1;
        if (M >= 100000) {
            free(pos);
            return -1;
        }
        if (next >= lim) {
            pos[M] = lim;
            break;
        }
        pos[M] = next;
        e = next;
        w = w * q;
    }
    if (2 * M + 1 > max_edges) {
        free(pos);
        return -1;
    }
    for (int j = 0; j <= M; ++j) {
        edges[M + j] = pos[j];
        edges[M - j] = -pos[j];
    }
    edges[M] = 0.0;
    free(pos);
    return 2 * M;
}

/* part of I(x,a) (App. A) other than the erf term */
static double o_I_rest(double x, double a)
{
    return -((2.0 * a) / O_SQRTPI) * lym1o_dawson(x) + ((a * a) * x) * exp(-(x * x));
}

/*
 * Bin-averaged Voigt profile over [xa, xb] in Doppler units (App. A):
 * <H> = [I(xb,a) - I(xa,a)] / dx_k.  The erf difference is taken through erfc
 * on the side away from line centre so that wing bins keep full precision.
 */
static double o_bin_H(double xa, double xb, double a, double dxk)
{
    double derf;
    if (xa >= 0.0)
        derf = (O_SQRTPI / 2.0) * (erfc(xa) - erfc(xb));
    else if (xb <= 0.0)
        derf = (O_SQRTPI / 2.0) * (erfc(-xb) - erfc(-xa));
    else
        derf = (O_SQRTPI / 2.0) * (erf(xb) - erf(xa));
    return (derf + (o_I_rest(xb, a) - o_I_rest(xa, a))) / dxk;
}

/*
 * Per-bin tables for n bins with the given dnu edges at temperature T:
 * dnu_k (width, Hz), nubar_k (absolute centre frequency, bin midpoint, App. A
 * footnote), Havg_k (bin-averaged Voigt), w_k (emitted fraction, from
 * phi_nu = H/sqrt(pi), renormalised to sum 1 so the grid conserves photons).
 * Returns eta = sum_k w_k Havg_k (the gray-group overlap factor).
 */
double lym1o_bin_tables(int n, const double *edges, double T, double *dnu, double *nubar,
                        double *Havg, double *w)
{
    double ln[3];
    lym1o_line(T, ln);
    double dnuD = ln[0], a = ln[1];
    double S = 0.0;
    for (int k = 0; k < n; ++k) {
        dnu[k] = edges[k + 1] - edges[k];
        nubar[k] = O_NU_LYA + 0.5 * (edges[k] + edges[k + 1]);
        double xa = edges[k] / dnuD, xb = edges[k + 1] / dnuD, dxk = dnu[k] / dnuD;
        Havg[k] = o_bin_H(xa, xb, a, dxk);
        w[k] = Havg[k] * dxk;
        S += w[k];
    }
    double eta = 0.0;
    for (int k = 0; k < n; ++k) {
        w[k] = w[k] / S;
        eta += w[k] * Havg[k];
    }
    return eta;
}

/* ======================================================================
 * Problem and context
 * ====================================================================== */
typedef struct {
    int nx, ny;          /* cells */
    int nbins;           /* bins of the frequency grid given by edges */
    int gray;            /* 1: one gray group (opacity alpha*eta), no step 3 */
    int recoil;          /* 1: atomic recoil in step 3 */
    int freq_step;       /* 1: run step 3 (ignored if gray) */
    double dx;           /* cell width (cm); the slab depth is also dx */
    double T;            /* gas temperature (K), uniform */
    double c_tilde;      /* (reduced) speed of light (cm/s) */
    double cfl;          /* CFL_RT (0.4 in the paper) */
    double kappa_abs;    /* dust absorption opacity kappa_ext(1-omega) (cm^2/g) */
    double kappa_F;      /* dust flux opacity kappa_ext(1-omega g) (cm^2/g) */
    const double *edges; /* nbins+1 ascending dnu edges (Hz) */
    const double *n_hi;  /* [ny][nx] cm^-3 */
    const double *rho_d; /* [ny][nx] g cm^-3 */
    const double *p_d;   /* [ny][nx] */
    const double *ux;    /* [ny][nx] cm/s */
    const double *uy;    /* [ny][nx] cm/s */
    const double *lum;   /* [ny][nx] erg/s emitted in the cell */
    int geometry;        /* 0: 2D Cartesian slab; 1: axisymmetric cylindrical (R = x, Z = y) with
                            the axis at R = 0 and the midplane at Z = 0 mirrored */
    int bc[4];           /* x-, x+, y-, y+ outflow kind: 0 = ghosts copy the edge cell
                            (zero gradient); 1 = outflow into vacuum (ghosts carry no
                            radiation; opacities and velocities are still copied); the
                            mirrored sides of geometry 1 ignore their entry */
    const double *temp;  /* [ny][nx] gas temperature (K) per cell, or NULL for the uniform T */
    /* Broad bands (Sec. 3, stellar and IR bands: the M1 moment equations per
     * band without frequency-derivative terms).  With band_aF set, nbins
     * counts bands, each a frequency-integrated group (dnu = 1, edges
     * ignored), step 3 is off, and the opacities and emission of each
     * [band][cell] are given: flux opacity alpha_F (cm^-1), absorption
     * opacity kappa (cm^-1) and emissivity j (erg s^-1 cm^-3 sr^-1).  The
     * Lya inputs (n_hi, rho_d, p_d, lum, temp) are not used. */
    const double *band_aF, *band_kap, *band_j;
    /* Active-bin pruning (Sec. 2.2): with prune > 0 a bin is advected only
     * while it holds more than prune of the Lya energy in the domain (the
     * paper's value is 1e-10), taken on the state at the start of the
     * substep; the other bins skip step 1 (fluxes, advection, work and hoop
     * terms) and still take steps 2 and 3.  0: every bin is advected. */
    double prune;
    /* Substep acceptance of step 2 (Sec. 2.1 step 2 and its footnote): 0 takes
     * one implicit emission/absorption update over dt (the default); 1
     * subcycles it per cell.  A trial substep of a cell is accepted when its
     * Lya energy density changes by |e'' - e'| / (e' + e_floor) < 0.1, with
     * e_floor = 4 pi J_floor / c and J_floor = 1e-15 erg cm^-2 s^-1 sr^-1;
     * otherwise the substep is halved and redone, until the accepted
     * substeps fill dt.  Readings (the paper gives the halving only): every
     * cell starts with the whole dt; after an accepted substep the next trial
     * doubles it (capped by what is left of dt); substeps are whole multiples
     * of dt / 2^40, one of that size is accepted whatever the change, and
     * after 2^16 trials in one substep every further trial is accepted (a
     * bound on the loop that finite inputs do not reach). */
    int accept;
} lym1o_problem;

typedef struct {
    double e_before, e_after;                  /* Lya energy in the domain, erg */
    double emitted, absorbed, outflow, work;   /* erg over the substep */
    double residual;                           /* e_after-e_before-(em-abs-out-work) */
    double max_f;                              /* max |H|/J after the substep */
    double n_unrealisable;                     /* (cell,bin) with |H| > J(1+1e-12) */
    double force_abs;                          /* sum |f| dV, dyn */
    double force_radial;                       /* sum f.rhat dV, dyn */
} lym1o_diag;

typedef struct {
    lym1o_problem p;
    int nb; /* state bins */
    double dnuD, a_v, sigma0, hkT, eta, dt_cfl, umax;
    double *dnu, *nubar, *Havg, *gem, *Rk, *half;
    double *alpha, *gxx, *gyy, *gsh;
    /* cylindrical geometry (per radian): R-face areas AR[nx+1], Z-face areas
     * AZ[nx], volumes Vol[nx], centroids Rbar[nx], centroid-to-face distances
     * dlL/dlR[nx+1] on the two sides of each R face, <1/R> = dR dZ / Vol,
     * full volumes 2 pi Vol, the emission factor w_k / (4 pi dnu_k) and
     * <u_R/R> per cell */
    double *AR, *AZ, *Vol, *Rbar, *dlL, *dlR, *invR, *V2pi, *gemc, *gphi;
    /* per-cell temperature (p.temp != NULL): <H>_k and the emission factor per
     * [k][cell] (A0 at the cell's T), the recoil factor h/(k_B T) and the
     * frequency-diffusion prefactor dnu_D^2/2 per cell; NULL otherwise */
    double *Hc, *Gc, *hkTc, *Kcc;
    /* emergent spectrum of the last substep (NULL: off): escaping energy (erg)
     * per [bin][outer face], faces ordered x- (j), x+ (j), y- (i), y+ (i) for
     * geometry 0 and R outer (j), Z outer (i) for geometry 1 */
    double *spec;
    /* accepted step-2 substeps of each cell in the last substep (NULL: not
     * recorded); only with p.accept */
    int *nsub;
} lym1o_ctx;

static int o_cl(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

/* 1 where index i lies beyond an edge whose outflow kind is vacuum */
static int o_vac(int i, int n, int bc_lo, int bc_hi)
{
    return (i < 0 && bc_lo == 1) || (i >= n && bc_hi == 1);
}

void lym1o_destroy(lym1o_ctx *c)
{
    if (!c) return;
    free(c->dnu); free(c->nubar); free(c->Havg); free(c->gem); free(c->Rk); free(c->half);
    free(c->alpha); free(c->gxx); free(c->gyy); free(c->gsh);
    free(c->AR); free(c->AZ); free(c->Vol); free(c->Rbar); free(c->dlL); free(c->dlR);
    free(c->invR); free(c->V2pi); free(c->gemc); free(c->gphi);
    free(c->Hc); free(c->Gc); free(c->hkTc); free(c->Kcc);
    free(c);
}

/* index along one axis with the low side mirrored (axis R = 0 or midplane
 * Z = 0) and the high side copied (outflow); *flip = 1 for a mirrored cell */
static int o_mir(int i, int n, int *flip)
{
    if (i < 0) {
        *flip = 1;
        return (-1 - i >= n) ? n - 1 : -1 - i;
    }
    *flip = 0;
    return i >= n ? n - 1 : i;
}

lym1o_ctx *lym1o_create(const lym1o_problem *p)
{
    if (p->nx < 1 || p->ny < 1 || p->nbins < 1 || p->dx <= 0.0) return NULL;
    for (int s = 0; s < 4; ++s)
        if (p->bc[s] != 0 && p->bc[s] != 1) return NULL;
    if (p->band_aF && (!p->band_kap || !p->band_j || p->gray || p->temp)) return NULL;
    /* the acceptance rule watches the Lya energy density: not for broad bands */
    if (p->accept != 0 && (p->accept != 1 || p->band_aF)) return NULL;
    lym1o_ctx *c = (lym1o_ctx *)calloc(1, sizeof *c);
    c->p = *p;
    if (p->band_aF) c->p.freq_step = 0;
    int nx = p->nx, ny = p->ny, N = p->nbins;
    double ln[3];
    lym1o_line(p->T, ln);
    c->dnuD = ln[0];
    c->a_v = ln[1];
    c->sigma0 = ln[2];
    c->hkT = O_HPL / (O_KB * p->T);
    double *dnu = malloc(N * sizeof(double)), *nub = malloc(N * sizeof(double));
    double *Hv = malloc(N * sizeof(double)), *w = malloc(N * sizeof(double));
    c->eta = p->band_aF ? 1.0 : lym1o_bin_tables(N, p->edges, p->T, dnu, nub, Hv, w);
    c->nb = p->gray ? 1 : N;
    int nb = c->nb;
    c->dnu = malloc(nb * sizeof(double));
    c->nubar = malloc(nb * sizeof(double));
    c->Havg = malloc(nb * sizeof(double));
    c->gem = malloc(nb * sizeof(double));
    c->Rk = malloc(nb * sizeof(double));
    c->half = malloc(nb * sizeof(double));
    double V = (p->dx * p->dx) * p->dx;
    double fourpiV = (4.0 * O_PI) * V;
    size_t nc = (size_t)nx * ny;
    if (p->gray) {
        c->dnu[0] = 1.0;
        c->nubar[0] = O_NU_LYA;
        c->Havg[0] = c->eta;
        c->gem[0] = 1.0 / fourpiV;
        c->Rk[0] = 0.0;
        c->half[0] = 0.5;
    } else if (p->band_aF) {
        for (int k = 0; k < N; ++k) {
            c->dnu[k] = 1.0;
            c->nubar[k] = O_NU_LYA;
            c->Havg[k] = 1.0;
            c->gem[k] = 0.0;
            c->Rk[k] = 0.0;
            c->half[k] = 0.5;
        }
    } else {
        for (int k = 0; k < N; ++k) {
            c->dnu[k] = dnu[k];
            c->nubar[k] = nub[k];
            c->Havg[k] = Hv[k];
            c->gem[k] = w[k] / (fourpiV * dnu[k]);
            c->Rk[k] = p->recoil ? (c->hkT - 2.0 / nub[k]) : 0.0;
            c->half[k] = 0.5 * dnu[k];
        }
    }
    free(dnu); free(nub); free(Hv); free(w);
    c->alpha = malloc(nc * sizeof(double));
    c->gxx = malloc(nc * sizeof(double));
    c->gyy = malloc(nc * sizeof(double));
    c->gsh = malloc(nc * sizeof(double));
    double umax = 0.0;
    if (p->geometry == 1) {
        const double dx = p->dx;
        c->AR = malloc((nx + 1) * sizeof(double));
        c->dlL = malloc((nx + 1) * sizeof(double));
        c->dlR = malloc((nx + 1) * sizeof(double));
        c->AZ = malloc(nx * sizeof(double));
        c->Vol = malloc(nx * sizeof(double));
        c->Rbar = malloc(nx * sizeof(double));
        c->invR = malloc(nx * sizeof(double));
        c->V2pi = malloc(nx * sizeof(double));
        c->gphi = malloc(nc * sizeof(double));
        c->gemc = malloc(nb * sizeof(double));
        for (int i = 0; i < nx; ++i) {
            double Rm = i * dx, Rp = (i + 1) * dx;
            c->AZ[i] = 0.5 * (Rp * Rp - Rm * Rm);
            c->Vol[i] = c->AZ[i] * dx;
            c->Rbar[i] = (2.0 / 3.0) * ((Rp * Rp * Rp - Rm * Rm * Rm) / (Rp * Rp - Rm * Rm));
            c->invR[i] = (dx * dx) / c->Vol[i];
            c->V2pi[i] = (2.0 * O_PI) * c->Vol[i];
        }
        for (int i = 0; i <= nx; ++i) {
            double Rf = i * dx;
            c->AR[i] = Rf * dx;
            double left = (i == 0) ? -c->Rbar[0] : c->Rbar[i - 1];
            double right = (i == nx) ? c->Rbar[nx - 1] + dx : c->Rbar[i];
            c->dlL[i] = Rf - left;
            c->dlR[i] = right - Rf;
        }
        if (p->gray) {
            c->gemc[0] = 1.0 / (4.0 * O_PI);
        } else if (p->band_aF) {
            for (int k = 0; k < N; ++k) c->gemc[k] = 0.0;
        } else {
            /* j_k = (L_cell / (2 pi Vol)) w_k / (4 pi dnu_k) */
            double *t1 = malloc(N * sizeof(double)), *t2 = malloc(N * sizeof(double));
            double *t3 = malloc(N * sizeof(double)), *t4 = malloc(N * sizeof(double));
            lym1o_bin_tables(N, p->edges, p->T, t1, t2, t3, t4);
            for (int k = 0; k < N; ++k) c->gemc[k] = t4[k] / ((4.0 * O_PI) * t1[k]);
            free(t1); free(t2); free(t3); free(t4);
        }
    }
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t id = (size_t)j * nx + i;
            c->alpha[id] = p->n_hi[id] * c->sigma0;
            if (p->temp) {
                double lc[3];
                lym1o_line(p->temp[id], lc);
                c->alpha[id] = p->n_hi[id] * lc[2];
            }
            if (p->geometry == 1) {
                /* mirrored ghosts: across the axis u_R flips, across the midplane u_Z flips */
                const double *ux = p->ux, *uy = p->uy;
                int fm, fp, gm, gp;
                int im = o_mir(i - 1, nx, &fm), ip = o_mir(i + 1, nx, &fp);
                int jm = o_mir(j - 1, ny, &gm), jp = o_mir(j + 1, ny, &gp);
                double uRm = ux[(size_t)j * nx + im] * (fm ? -1.0 : 1.0);
                double uRp = ux[(size_t)j * nx + ip];
                double uZm = uy[(size_t)jm * nx + i] * (gm ? -1.0 : 1.0);
                double uZp = uy[(size_t)jp * nx + i];
                double uZl = uy[(size_t)j * nx + im], uZr = uy[(size_t)j * nx + ip];
                double uRd = ux[(size_t)jm * nx + i], uRu = ux[(size_t)jp * nx + i];
                double h2 = 2.0 * p->dx;
                c->gxx[id] = (uRp - uRm) / h2;
                c->gyy[id] = (uZp - uZm) / h2;
                c->gsh[id] = (uRu - uRd) / h2 + (uZr - uZl) / h2;
                /* <u_R / R> from the face velocities (mean of the two cells) */
                double fL = 0.5 * (uRm + ux[id]), fR = 0.5 * (ux[id] + uRp);
                c->gphi[id] = (fR + fL) / ((i + 1) * p->dx + i * p->dx);
                double um = sqrt(ux[id] * ux[id] + uy[id] * uy[id]);
                if (um > umax) umax = um;
                continue;
            }
            const double *ux = p->ux, *uy = p->uy;
            size_t xm = (size_t)j * nx + o_cl(i - 1, nx), xp = (size_t)j * nx + o_cl(i + 1, nx);
            size_t ym = (size_t)o_cl(j - 1, ny) * nx + i, yp = (size_t)o_cl(j + 1, ny) * nx + i;
            double h2 = 2.0 * p->dx;
            c->gxx[id] = (ux[xp] - ux[xm]) / h2;
            c->gyy[id] = (uy[yp] - uy[ym]) / h2;
            c->gsh[id] = (ux[yp] - ux[ym]) / h2 + (uy[xp] - uy[xm]) / h2;
            double um = sqrt(ux[id] * ux[id] + uy[id] * uy[id]);
            if (um > umax) umax = um;
        }
    /* RT time step (Sec. 2.1, CFL condition, D = 2 dimensions) */
    c->dt_cfl = (p->cfl / 2.0) * (p->dx / (p->c_tilde + umax));
    c->umax = umax;
    if (p->temp) {
        /* A0 at every cell's own temperature (App. A: <H>_k, the Doppler width
         * and a_v at T; Sec. 2.1 step 2: emission fractions) */
        c->Hc = malloc((size_t)nb * nc * sizeof(double));
        c->Gc = malloc((size_t)nb * nc * sizeof(double));
        c->hkTc = malloc(nc * sizeof(double));
        c->Kcc = malloc(nc * sizeof(double));
        double *d1 = malloc(N * sizeof(double)), *d2 = malloc(N * sizeof(double));
        double *d3 = malloc(N * sizeof(double)), *d4 = malloc(N * sizeof(double));
        for (size_t id = 0; id < nc; ++id) {
            const double Tc = p->temp[id];
            double lc[3];
            lym1o_line(Tc, lc);
            c->hkTc[id] = O_HPL / (O_KB * Tc);
            c->Kcc[id] = 0.5 * (lc[0] * lc[0]);
            double etac = lym1o_bin_tables(N, p->edges, Tc, d1, d2, d3, d4);
            int i = (int)(id % nx);
            for (int k = 0; k < nb; ++k) {
                size_t kid = (size_t)k * nc + id;
                if (p->gray) {
                    c->Hc[kid] = etac;
                    c->Gc[kid] = (p->geometry == 1) ? 1.0 / (4.0 * O_PI) : 1.0 / fourpiV;
                } else {
                    c->Hc[kid] = d3[k];
                    c->Gc[kid] = (p->geometry == 1) ? d4[k] / ((4.0 * O_PI) * d1[k])
                                                    : d4[k] / (fourpiV * d1[k]);
                }
            }
            (void)i;
        }
        free(d1); free(d2); free(d3); free(d4);
    }
    return c;
}

double lym1o_dt_cfl(const lym1o_ctx *c) { return c->dt_cfl; }
double lym1o_eta(const lym1o_ctx *c) { return c->eta; }
int lym1o_nb(const lym1o_ctx *c) { return c->nb; }
void lym1o_tables(const lym1o_ctx *c, double *dnu, double *nubar, double *Havg, double *gem)
{
    for (int k = 0; k < c->nb; ++k) {
        dnu[k] = c->dnu[k];
        nubar[k] = c->nubar[k];
        Havg[k] = c->Havg[k];
        gem[k] = c->gem[k];
    }
}

/* ======================================================================
 * A1: closure and reconstruction helpers
 * ====================================================================== */
/* Levermore M1 closure (Sec. 2.1): D = (1-chi)/2 I + (3chi-1)/2 h h, returns
 * the normal-normal and normal-tangential components for f = (fn, ft). */
static void o_closure(double fn, double ft, double *Dnn, double *Dnt, double *Dtt)
{
    double f2 = fn * fn + ft * ft;
    double chi = (3.0 + 4.0 * f2) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f2));
    double dA = (1.0 - chi) / 2.0, dB = (3.0 * chi - 1.0) / 2.0;
    if (f2 > 0.0) {
        *Dnn = dA + (dB * (fn * fn)) / f2;
        *Dnt = (dB * (fn * ft)) / f2;
        *Dtt = dA + (dB * (ft * ft)) / f2;
    } else {
        *Dnn = dA;
        *Dnt = 0.0;
        *Dtt = dA;
    }
}

void lym1o_closure(double fx, double fy, double *D3 /* Dxx, Dxy, Dyy */)
{
    o_closure(fx, fy, &D3[0], &D3[1], &D3[2]);
}

/* interpolation factor between GLF and diffusion fluxes (Sec. 2.1) */
double lym1o_eps(double tau) { return (0.2 + tau) / ((0.2 + tau) + tau * tau); }

/* Step 3 leaves every cell causal (Sec. 2.1 step 3: |H|/J <= 1 with H
 * rescaled by J_new/J_old): an H longer than J is shortened to J along its
 * direction, and H = 0 where J <= 0. */
static void o_causal(double J, double *Hx, double *Hy)
{
    double hn = sqrt((*Hx) * (*Hx) + (*Hy) * (*Hy));
    if (hn > J) {
        if (J > 0.0) {
            double s = J / hn;
            *Hx = (*Hx) * s;
            *Hy = (*Hy) * s;
        } else {
            *Hx = 0.0;
            *Hy = 0.0;
        }
    }
}

static double o_minmod(double a, double b)
{
    if (a > 0.0 && b > 0.0) return a < b ? a : b;
    if (a < 0.0 && b < 0.0) return a > b ? a : b;
    return 0.0;
}

/* primitive state of one cell: J and the reduced flux components (n, t) */
typedef struct { double J, fn, ft; } o_prim;

static o_prim o_make_prim(double J, double Hn, double Ht)
{
    o_prim q;
    q.J = J;
    if (J > 0.0) {
        q.fn = Hn / J;
        q.ft = Ht / J;
    } else {
        q.fn = 0.0;
        q.ft = 0.0;
    }
    return q;
}

/*
 * A1+A2: flux across the face between cells "0" and "1" (normal direction n,
 * tangential t).  qm, q0, q1, q2 are the cells at offsets -1, 0, +1, +2 along
 * the normal.  Returns the flux of J (FJ), of H_n (Fn) and of H_t (Ft).
 */
static void o_face(o_prim qm, o_prim q0, o_prim q1, o_prim q2, double aF0, double aF1,
                   double un0, double un1, double dl0, double dl1, double *FJ, double *Fn,
                   double *Ft)
{
    /* MinMod-limited linear reconstruction of J, f_n, f_t */
    double sJ0 = o_minmod(q0.J - qm.J, q1.J - q0.J), sJ1 = o_minmod(q1.J - q0.J, q2.J - q1.J);
    double sn0 = o_minmod(q0.fn - qm.fn, q1.fn - q0.fn), sn1 = o_minmod(q1.fn - q0.fn, q2.fn - q1.fn);
    double st0 = o_minmod(q0.ft - qm.ft, q1.ft - q0.ft), st1 = o_minmod(q1.ft - q0.ft, q2.ft - q1.ft);
    double JL = q0.J + 0.5 * sJ0, fnL = q0.fn + 0.5 * sn0, ftL = q0.ft + 0.5 * st0;
    double JR = q1.J - 0.5 * sJ1, fnR = q1.fn - 0.5 * sn1, ftR = q1.ft - 0.5 * st1;
    /* |f| > 1 at the interface: scale the components down */
    double f2L = fnL * fnL + ftL * ftL;
    if (f2L > 1.0) {
        double r = sqrt(f2L);
        fnL = fnL / r;
        ftL = ftL / r;
    }
    double f2R = fnR * fnR + ftR * ftR;
    if (f2R > 1.0) {
        double r = sqrt(f2R);
        fnR = fnR / r;
        ftR = ftR / r;
    }
    double HnL = JL * fnL, HtL = JL * ftL, HnR = JR * fnR, HtR = JR * ftR;
    double DnnL, DntL, DttL, DnnR, DntR, DttR;
    o_closure(fnL, ftL, &DnnL, &DntL, &DttL);
    o_closure(fnR, ftR, &DnnR, &DntR, &DttR);
    double KnnL = DnnL * JL, KntL = DntL * JL, KnnR = DnnR * JR, KntR = DntR * JR;
    /* flux optical depth: alpha_F times the centroid-to-face distance on each side */
    double tau = aF0 * dl0 + aF1 * dl1;
    double eps = (0.2 + tau) / ((0.2 + tau) + tau * tau);
    double dif = (tau > 0.0) ? ((1.0 - eps) * (q1.J - q0.J)) / (3.0 * tau) : 0.0;
    /* corrected GLF flux for J, modified GLF flux for K */
    double fJ = (eps * (0.5 * (HnL + HnR)) - eps * (0.5 * (JR - JL))) - dif;
    double fn = 0.5 * (KnnL + KnnR) - eps * (0.5 * (HnR - HnL));
    double ft = 0.5 * (KntL + KntR) - eps * (0.5 * (HtR - HtL));
    /* upwind advection of uJ/c and uH/c with the face velocity */
    double uf = 0.5 * (un0 + un1);
    if (uf > 0.0) {
        fJ = fJ + (uf * JL) / O_C;
        fn = fn + (uf * HnL) / O_C;
        ft = ft + (uf * HtL) / O_C;
    } else if (uf < 0.0) {
        fJ = fJ + (uf * JR) / O_C;
        fn = fn + (uf * HnR) / O_C;
        ft = ft + (uf * HtR) / O_C;
    }
    *FJ = fJ;
    *Fn = fn;
    *Ft = ft;
}

/* exported for unit pins: flux across one face from 4 cells along the normal */
void lym1o_face_flux(const double *J4, const double *Hn4, const double *Ht4, double aF0, double aF1,
                     double un0, double un1, double dx, double *out3)
{
    o_prim q[4];
    for (int m = 0; m < 4; ++m) q[m] = o_make_prim(J4[m], Hn4[m], Ht4[m]);
    o_face(q[0], q[1], q[2], q[3], aF0, aF1, un0, un1, 0.5 * dx, 0.5 * dx, &out3[0], &out3[1],
           &out3[2]);
}

/* ======================================================================
 * A6: frequency step for one cell (App. A)
 * ====================================================================== */
/*
 * Solves (J_k - Jin_k)/(ct dt) = F+_k J_{k+1} - F_k J_k + F-_k J_{k-1} with
 * zero-flux ends, K_k = dnuD^2 alpha <H>_k / 2, C_k = K_k R_k + (nubar_k/c)
 * DdU_k, P_k = C_k dlt_k / K_k (dlt_k = half bin width, midpoint centres).
 *
 * Leakage coefficients (App. A) written per interface k+1/2 as
 *   A = (1 - phiL(P_k)) / den,   B = (1 - phiR(P_{k+1})) / den,
 *   den = chiL(P_k) dlt_k/K_k - chiR(P_{k+1}) dlt_{k+1}/K_{k+1},
 * so that dnu_k F+_k = B_{k+1/2}, dnu_k F-_k = A_{k-1/2},
 * dnu_k F_k = A_{k+1/2} + B_{k-1/2}.  With E(z) = expm1(z)/z (z <= 0, E(0) = 1):
 *   chiL(P) = exp(max(-P,0)) E(-|P|),  -chiR(P) = exp(max(P,0)) E(-|P|),
 * and the common factor exp(m), m = max(0, -P_k, P_{k+1}), is divided out of
 * numerators and denominator, so all exponentials have non-positive arguments.
 *
 * Elimination in conservative form (row k times dnu_k, s_k = dnu_k/(ct dt)):
 *   (s_k + A_{k+1/2} + B_{k-1/2}) J_k - B_{k+1/2} J_{k+1} - A_{k-1/2} J_{k-1} = s_k Jin_k.
 * Forward: E_0 = s_0, E_k = s_k + B_{k-1/2} q_{k-1}, D'_k = E_k + A_{k+1/2},
 *   r_k = s_k Jin_k + A_{k-1/2} g_{k-1}, with inv = 1/D'_k, q_k = E_k inv,
 *   g_k = r_k inv, h_k = B_{k+1/2} inv.
 * Back: J_{N-1} = g_{N-1}, J_k = g_k + h_k J_{k+1}.
 * Every quantity is a sum or product of non-negative terms for Jin >= 0.
 */
static void o_freq_cell(int N, const double *dnu, const double *half, const double *Havg,
                        const double *Rk, const double *nubar_c, double Kc, const double *DdU,
                        double cdt, const double *Jin, double *Jout, double *scr /* 6N */)
{
    double *P = scr, *a = scr + N, *e = scr + 2 * N, *g = scr + 3 * N, *hh = scr + 4 * N;
    for (int k = 0; k < N; ++k) {
        double K = Kc * Havg[k];
        double C = K * Rk[k] + nubar_c[k] * DdU[k];
        P[k] = (C * half[k]) / K;
        a[k] = half[k] / K;
        double z = -fabs(P[k]);
        e[k] = (z == 0.0) ? 1.0 : lym1o_expm1(z) / z;
    }
    double Eprev = 0.0, qprev = 0.0, gprev = 0.0, Bprev = 0.0, Aprev = 0.0;
    for (int k = 0; k < N; ++k) {
        double Ak = 0.0, Bk = 0.0; /* interface k+1/2 */
        if (k + 1 < N) {
            double p = P[k], q = P[k + 1];
            double d1 = (-p > 0.0) ? -p : 0.0, d2 = (q > 0.0) ? q : 0.0;
            double m = (d1 > d2) ? d1 : d2;
            double den = lym1o_exp(d1 - m) * (e[k] * a[k]) + lym1o_exp(d2 - m) * (e[k + 1] * a[k + 1]);
            Ak = lym1o_exp(-p - m) / den;
            Bk = lym1o_exp(q - m) / den;
        }
        double s = dnu[k] / cdt;
        double E = (k == 0) ? s : s + Bprev * qprev;
        double r = (k == 0) ? s * Jin[k] : s * Jin[k] + Aprev * gprev;
        double Dp = E + Ak;
        double inv = 1.0 / Dp;
        g[k] = r * inv;
        hh[k] = Bk * inv;
        qprev = E * inv;
        gprev = g[k];
        Eprev = E;
        Bprev = Bk;
        Aprev = Ak;
    }
    (void)Eprev;
    Jout[N - 1] = g[N - 1];
    for (int k = N - 2; k >= 0; --k) Jout[k] = g[k] + hh[k] * Jout[k + 1];
}

/* exported for pins: one cell's frequency step with given per-bin D:grad(u) */
void lym1o_freq_solve(int N, const double *edges, double T, double alpha, int recoil,
                      const double *DdU, double cdt, const double *Jin, double *Jout)
{
    double ln[3];
    lym1o_line(T, ln);
    double *dnu = malloc(N * sizeof(double)), *nub = malloc(N * sizeof(double));
    double *Hv = malloc(N * sizeof(double)), *w = malloc(N * sizeof(double));
    double *half = malloc(N * sizeof(double)), *Rk = malloc(N * sizeof(double));
    double *nbc = malloc(N * sizeof(double)), *scr = malloc(6 * N * sizeof(double));
    lym1o_bin_tables(N, edges, T, dnu, nub, Hv, w);
    double hkT = O_HPL / (O_KB * T);
    for (int k = 0; k < N; ++k) {
        half[k] = 0.5 * dnu[k];
        Rk[k] = recoil ? (hkT - 2.0 / nub[k]) : 0.0;
        nbc[k] = nub[k] / O_C;
    }
    double Kc = (0.5 * (ln[0] * ln[0])) * alpha;
    o_freq_cell(N, dnu, half, Hv, Rk, nbc, Kc, DdU, cdt, Jin, Jout, scr);
    free(dnu); free(nub); free(Hv); free(w); free(half); free(Rk); free(nbc); free(scr);
}

/* exported for pins: leakage coefficients A_{k+1/2}, B_{k+1/2} (N-1 each) */
void lym1o_leakage(int N, const double *edges, double T, double alpha, int recoil,
                   const double *DdU, double *Aout, double *Bout)
{
    double ln[3];
    lym1o_line(T, ln);
    double *dnu = malloc(N * sizeof(double)), *nub = malloc(N * sizeof(double));
    double *Hv = malloc(N * sizeof(double)), *w = malloc(N * sizeof(double));
    double *P = malloc(N * sizeof(double)), *a = malloc(N * sizeof(double)), *e = malloc(N * sizeof(double));
    lym1o_bin_tables(N, edges, T, dnu, nub, Hv, w);
    double hkT = O_HPL / (O_KB * T);
    double Kc = (0.5 * (ln[0] * ln[0])) * alpha;
    for (int k = 0; k < N; ++k) {
        double half = 0.5 * dnu[k], K = Kc * Hv[k];
        double Rk = recoil ? (hkT - 2.0 / nub[k]) : 0.0;
        double C = K * Rk + (nub[k] / O_C) * DdU[k];
        P[k] = (C * half) / K;
        a[k] = half / K;
        double z = -fabs(P[k]);
        e[k] = (z == 0.0) ? 1.0 : lym1o_expm1(z) / z;
    }
    for (int k = 0; k + 1 < N; ++k) {
        double p = P[k], q = P[k + 1];
        double d1 = (-p > 0.0) ? -p : 0.0, d2 = (q > 0.0) ? q : 0.0;
        double m = (d1 > d2) ? d1 : d2;
        double den = lym1o_exp(d1 - m) * (e[k] * a[k]) + lym1o_exp(d2 - m) * (e[k + 1] * a[k + 1]);
        Aout[k] = lym1o_exp(-p - m) / den;
        Bout[k] = lym1o_exp(q - m) / den;
    }
    free(dnu); free(nub); free(Hv); free(w); free(P); free(a); free(e);
}

/* ======================================================================
 * Neumaier compensated sum
 * ====================================================================== */
typedef struct { double s, c; } o_ksum;
static void o_kadd(o_ksum *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v))
        a->c += (a->s - t) + v;
    else
        a->c += (v - t) + a->s;
    a->s = t;
}
static double o_kval(const o_ksum *a) { return a->s + a->c; }

/* Active bins of a substep (Sec. 2.2): E_k = dnu_k sum_cells w J_k (w: the
 * cell volume up to a constant), active while E_k > prune sum_k E_k.  NULL
 * when pruning is off. */
static unsigned char *o_active_bins(const lym1o_ctx *c, const double *J)
{
    const lym1o_problem *p = &c->p;
    if (!(p->prune > 0.0)) return NULL;
    const int nb = c->nb, nx = p->nx;
    const size_t nc = (size_t)nx * p->ny;
    double *E = malloc(nb * sizeof(double));
    o_ksum tot = {0.0, 0.0};
    for (int k = 0; k < nb; ++k) {
        o_ksum s = {0.0, 0.0};
        for (size_t id = 0; id < nc; ++id) {
            const double w = p->geometry == 1 ? c->V2pi[id % nx] : 1.0;
            o_kadd(&s, w * J[(size_t)k * nc + id]);
        }
        E[k] = c->dnu[k] * o_kval(&s);
        o_kadd(&tot, E[k]);
    }
    unsigned char *a = malloc(nb);
    const double cut = p->prune * o_kval(&tot);
    for (int k = 0; k < nb; ++k) a[k] = E[k] > cut;
    free(E);
    return a;
}

static void o_zero(double *a, size_t n)
{
    for (size_t i = 0; i < n; ++i) a[i] = 0.0;
}

static double o_energy(const lym1o_ctx *c, const double *J)
{
    size_t nc = (size_t)c->p.nx * c->p.ny;
    o_ksum S = {0.0, 0.0};
    for (int k = 0; k < c->nb; ++k)
        for (size_t id = 0; id < nc; ++id) o_kadd(&S, c->dnu[k] * J[(size_t)k * nc + id]);
    double V = (c->p.dx * c->p.dx) * c->p.dx;
    return ((4.0 * O_PI) / O_C) * V * o_kval(&S);
}

double lym1o_energy(const lym1o_ctx *c, const double *J) { return o_energy(c, J); }

/* ======================================================================
 * One substep of length dt: state (J, Hx, Hy) [k][y][x] -> (Jo, Hxo, Hyo),
 * force (fx, fy) [y][x] in dyn cm^-3.  Input and output may not alias.
 * ====================================================================== */
int lym1o_substep_cyl(const lym1o_ctx *c, double dt, const double *J, const double *Hx,
                      const double *Hy, double *Jo, double *Hxo, double *Hyo, double *fx,
                      double *fy, lym1o_diag *dg);

/* per-bin table entry, or the cell's own entry under a temperature field */
#define HAV(k, id) (c->Hc ? c->Hc[(size_t)(k) * nc + (id)] : c->Havg[k])
#define GEMK(k, id) (c->Gc ? c->Gc[(size_t)(k) * nc + (id)] : c->gem[k])
#define GEMC(k, id) (c->Gc ? c->Gc[(size_t)(k) * nc + (id)] : c->gemc[k])
/* a band's own [band][cell] input */
#define BND(a, k, id) (p->a[(size_t)(k) * nc + (id)])

/* step 3 of one cell: the per-bin tables or the cell's own (temperature field) */
static void o_freq_of_cell(const lym1o_ctx *c, size_t id, size_t nc, const double *nbc,
                           const double *DdU, double cdt, const double *Jin, double *Jn,
                           double *scr, double *Hcell, double *Rcell)
{
    const int nb = c->nb;
    if (!c->Hc) {
        const double Kc0 = 0.5 * (c->dnuD * c->dnuD);
        o_freq_cell(nb, c->dnu, c->half, c->Havg, c->Rk, nbc, Kc0 * c->alpha[id], DdU, cdt, Jin, Jn,
                    scr);
        return;
    }
    for (int k = 0; k < nb; ++k) {
        Hcell[k] = c->Hc[(size_t)k * nc + id];
        Rcell[k] = c->p.recoil ? (c->hkTc[id] - 2.0 / c->nubar[k]) : 0.0;
    }
    o_freq_cell(nb, c->dnu, c->half, Hcell, Rcell, nbc, c->Kcc[id] * c->alpha[id], DdU, cdt, Jin, Jn,
                scr);
}

/* Step 2 of one cell with the substep acceptance rule (Sec. 2.1 step 2, see
 * lym1o_problem.accept), in place on the cell's post-transport state
 * (Jo, Hxo, Hyo).  Each accepted substep of length h is the printed implicit
 * update J'' = (J' + c h j)/(1 + c h kappa), H'' = H'/(1 + c h alpha_F); the
 * force sum dnu (H' - H''), the emission dnu c h j and the absorption
 * dnu c h kappa J'' add up over the accepted substeps.  vol weights the
 * emission and absorption (1 for geometry 0, the ring volume 2 pi Vol for
 * geometry 1); jfac turns the cell's emission factor into j (lum for geometry
 * 0, lum / (2 pi Vol) for geometry 1). */
#define O_SUB_LEVELS 40
#define O_SUB_MAX_TRIALS 65536
#define O_J_FLOOR 1e-15
static int o_step2_subcycle(const lym1o_ctx *c, size_t id, size_t nc, double dt, double jfac,
                            int cyl, double *Jo, double *Hxo, double *Hyo, double *ax, double *ay,
                            double *em, double *ab)
{
    const lym1o_problem *p = &c->p;
    const int nb = c->nb;
    const long long full = 1LL << O_SUB_LEVELS;
    long long done = 0, size = full;
    int n = 0, trials = 0;
    double e_cur = 0.0;
    for (int k = 0; k < nb; ++k) e_cur = e_cur + c->dnu[k] * Jo[(size_t)k * nc + id];
    while (done < full) {
        if (size > full - done) size = full - done;
        const double h = dt * ((double)size / (double)full);
        const double ch = p->c_tilde * h;
        ++trials;
        /* trial: the energy density after this substep (in units of 4 pi / c) */
        double e_new = 0.0;
        for (int k = 0; k < nb; ++k) {
            const double aH = c->alpha[id] * HAV(k, id);
            const double kap = p->rho_d[id] * p->kappa_abs + p->p_d[id] * aH;
            const double js = jfac * (cyl ? GEMC(k, id) : GEMK(k, id));
            const double Jt = (Jo[(size_t)k * nc + id] + ch * js) / (1.0 + ch * kap);
            e_new = e_new + c->dnu[k] * Jt;
        }
        const double change = fabs(e_new - e_cur) / (e_cur + O_J_FLOOR);
        if (!(change < 0.1) && size > 1 && trials <= O_SUB_MAX_TRIALS) {
            size = size / 2;
            continue;
        }
        for (int k = 0; k < nb; ++k) {
            const size_t kid = (size_t)k * nc + id;
            const double aH = c->alpha[id] * HAV(k, id);
            const double kap = p->rho_d[id] * p->kappa_abs + p->p_d[id] * aH;
            const double aF = aH + p->rho_d[id] * p->kappa_F;
            const double js = jfac * (cyl ? GEMC(k, id) : GEMK(k, id));
            const double J2 = (Jo[kid] + ch * js) / (1.0 + ch * kap);
            const double Hx2 = Hxo[kid] / (1.0 + ch * aF);
            const double Hy2 = Hyo[kid] / (1.0 + ch * aF);
            ax[id] = ax[id] + c->dnu[k] * (Hxo[kid] - Hx2);
            ay[id] = ay[id] + c->dnu[k] * (Hyo[kid] - Hy2);
            em[id] = em[id] + c->dnu[k] * (ch * js);
            ab[id] = ab[id] + c->dnu[k] * (ch * (kap * J2));
            Jo[kid] = J2;
            Hxo[kid] = Hx2;
            Hyo[kid] = Hy2;
        }
        e_cur = e_new;
        done += size;
        ++n;
        size = size * 2;
    }
    return n;
}

int lym1o_substep(const lym1o_ctx *c, double dt, const double *J, const double *Hx,
                  const double *Hy, double *Jo, double *Hxo, double *Hyo, double *fx,
                  double *fy, lym1o_diag *dg)
{
    if (c->p.geometry == 1) return lym1o_substep_cyl(c, dt, J, Hx, Hy, Jo, Hxo, Hyo, fx, fy, dg);
    const lym1o_problem *p = &c->p;
    const int nx = p->nx, ny = p->ny, nb = c->nb;
    const size_t nc = (size_t)nx * ny;
    const double dx = p->dx, half_dx = 0.5 * dx, cdt = p->c_tilde * dt;
    const double V = (dx * dx) * dx;
    const double eunit = ((4.0 * O_PI) / O_C) * V; /* erg per (Hz-weighted J) per cell */
    lym1o_diag d;
    memset(&d, 0, sizeof d);
    d.e_before = o_energy(c, J);
    o_ksum s_em = {0, 0}, s_ab = {0, 0}, s_out = {0, 0}, s_wk = {0, 0};

    /* per-bin work arrays */
    double *FJx = malloc((size_t)(nx + 1) * ny * sizeof(double));
    double *FHxx = malloc((size_t)(nx + 1) * ny * sizeof(double));
    double *FHyx = malloc((size_t)(nx + 1) * ny * sizeof(double));
    double *FJy = malloc((size_t)nx * (ny + 1) * sizeof(double));
    double *FHxy = malloc((size_t)nx * (ny + 1) * sizeof(double));
    double *FHyy = malloc((size_t)nx * (ny + 1) * sizeof(double));
    double *Wk = malloc(nc * sizeof(double));
    double *ax = malloc(nc * sizeof(double)), *ay = malloc(nc * sizeof(double));
    for (size_t id = 0; id < nc; ++id) {
        ax[id] = 0.0;
        ay[id] = 0.0;
    }
    unsigned char *act = o_active_bins(c, J);

    for (int k = 0; k < nb; ++k) {
        const double *Jk = J + (size_t)k * nc, *Hxk = Hx + (size_t)k * nc, *Hyk = Hy + (size_t)k * nc;
#define AF(id) (p->band_aF ? BND(band_aF, k, id) : c->alpha[id] * HAV(k, id) + p->rho_d[id] * p->kappa_F)
        const int on = !act || act[k]; /* pruned bins: no step 1 */
        if (!on) {
            o_zero(FJx, (size_t)(nx + 1) * ny);
            o_zero(FHxx, (size_t)(nx + 1) * ny);
            o_zero(FHyx, (size_t)(nx + 1) * ny);
            o_zero(FJy, (size_t)nx * (ny + 1));
            o_zero(FHxy, (size_t)nx * (ny + 1));
            o_zero(FHyy, (size_t)nx * (ny + 1));
        } else {
        /* x faces: face i sits between cells i-1 and i, i = 0..nx */
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                o_prim q[4];
                for (int m = 0; m < 4; ++m) {
                    int ii = i - 2 + m;
                    size_t id = (size_t)j * nx + o_cl(ii, nx);
                    q[m] = o_vac(ii, nx, p->bc[0], p->bc[1]) ? o_make_prim(0.0, 0.0, 0.0)
                                                              : o_make_prim(Jk[id], Hxk[id], Hyk[id]);
                }
                size_t i0 = (size_t)j * nx + o_cl(i - 1, nx), i1 = (size_t)j * nx + o_cl(i, nx);
                size_t f = (size_t)j * (nx + 1) + i;
                o_face(q[0], q[1], q[2], q[3], AF(i0), AF(i1), p->ux[i0], p->ux[i1], half_dx, half_dx,
                       &FJx[f], &FHxx[f], &FHyx[f]);
            }
        /* y faces: face j sits between rows j-1 and j, j = 0..ny */
#pragma omp parallel for schedule(static)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i < nx; ++i) {
                o_prim q[4];
                for (int m = 0; m < 4; ++m) {
                    int jj = j - 2 + m;
                    size_t id = (size_t)o_cl(jj, ny) * nx + i;
                    q[m] = o_vac(jj, ny, p->bc[2], p->bc[3]) ? o_make_prim(0.0, 0.0, 0.0)
                                                              : o_make_prim(Jk[id], Hyk[id], Hxk[id]);
                }
                size_t i0 = (size_t)o_cl(j - 1, ny) * nx + i, i1 = (size_t)o_cl(j, ny) * nx + i;
                size_t f = (size_t)j * nx + i;
                o_face(q[0], q[1], q[2], q[3], AF(i0), AF(i1), p->uy[i0], p->uy[i1], half_dx, half_dx,
                       &FJy[f], &FHyy[f], &FHxy[f]);
            }
        }
        /* A3 explicit update, A4 implicit source, A5 force accumulation */
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t id = (size_t)j * nx + i, kid = (size_t)k * nc + id;
                o_prim q = o_make_prim(Jk[id], Hxk[id], Hyk[id]);
                double fxc = q.fn, fyc = q.ft, f2 = fxc * fxc + fyc * fyc;
                if (f2 > 1.0) {
                    double r = sqrt(f2);
                    fxc = fxc / r;
                    fyc = fyc / r;
                }
                double Dxx, Dxy, Dyy;
                o_closure(fxc, fyc, &Dxx, &Dxy, &Dyy);
                double W = ((Dxx * Jk[id]) * c->gxx[id] + (Dyy * Jk[id]) * c->gyy[id]) +
                           (Dxy * Jk[id]) * c->gsh[id];
                if (!on) W = 0.0;
                Wk[id] = W;
                size_t fxl = (size_t)j * (nx + 1) + i, fyl = (size_t)j * nx + i;
                double divJ = (FJx[fxl + 1] - FJx[fxl]) + (FJy[fyl + nx] - FJy[fyl]);
                double divHx = (FHxx[fxl + 1] - FHxx[fxl]) + (FHxy[fyl + nx] - FHxy[fyl]);
                double divHy = (FHyx[fxl + 1] - FHyx[fxl]) + (FHyy[fyl + nx] - FHyy[fyl]);
                double J1 = Jk[id] - cdt * (divJ / dx + W / O_C);
                double Hx1 = Hxk[id] - cdt * (divHx / dx);
                double Hy1 = Hyk[id] - cdt * (divHy / dx);
                /* A4: (J''-J')/(ct dt) = j - kappa J'', (H''-H')/(ct dt) = -aF H'' */
                double aH = c->alpha[id] * HAV(k, id);
                double kap = p->rho_d[id] * p->kappa_abs + p->p_d[id] * aH;
                double aF = aH + p->rho_d[id] * p->kappa_F;
                double js = p->lum[id] * GEMK(k, id);
                if (p->band_aF) {
                    kap = BND(band_kap, k, id);
                    aF = BND(band_aF, k, id);
                    js = BND(band_j, k, id);
                }
                if (p->accept) { /* step 2 is subcycled per cell after the bin loop */
                    Jo[kid] = J1;
                    Hxo[kid] = Hx1;
                    Hyo[kid] = Hy1;
                    continue;
                }
                double J2 = (J1 + cdt * js) / (1.0 + cdt * kap);
                double Hx2 = Hx1 / (1.0 + cdt * aF);
                double Hy2 = Hy1 / (1.0 + cdt * aF);
                Jo[kid] = J2;
                Hxo[kid] = Hx2;
                Hyo[kid] = Hy2;
                ax[id] = ax[id] + c->dnu[k] * (Hx1 - Hx2);
                ay[id] = ay[id] + c->dnu[k] * (Hy1 - Hy2);
            }
        /* bookkeeping for this bin (serial, fixed order) */
        for (size_t id = 0; id < nc; ++id) {
            size_t kid = (size_t)k * nc + id;
            double aH = c->alpha[id] * HAV(k, id);
            double kap = p->rho_d[id] * p->kappa_abs + p->p_d[id] * aH;
            double js = p->lum[id] * GEMK(k, id);
            if (p->band_aF) {
                kap = BND(band_kap, k, id);
                js = BND(band_j, k, id);
            }
            if (!p->accept) {
                o_kadd(&s_em, c->dnu[k] * (cdt * js));
                o_kadd(&s_ab, c->dnu[k] * (cdt * (kap * Jo[kid])));
            }
            o_kadd(&s_wk, c->dnu[k] * (cdt * (Wk[id] / O_C)));
        }
        const int nf = 2 * (nx + ny);
        for (int j = 0; j < ny; ++j) {
            double lo = c->dnu[k] * (cdt * (-FJx[(size_t)j * (nx + 1)] / dx));
            double hi = c->dnu[k] * (cdt * (FJx[(size_t)j * (nx + 1) + nx] / dx));
            o_kadd(&s_out, lo);
            o_kadd(&s_out, hi);
            if (c->spec) {
                c->spec[(size_t)k * nf + j] = eunit * lo;
                c->spec[(size_t)k * nf + ny + j] = eunit * hi;
            }
        }
        for (int i = 0; i < nx; ++i) {
            double lo = c->dnu[k] * (cdt * (-FJy[i] / dx));
            double hi = c->dnu[k] * (cdt * (FJy[(size_t)ny * nx + i] / dx));
            o_kadd(&s_out, lo);
            o_kadd(&s_out, hi);
            if (c->spec) {
                c->spec[(size_t)k * nf + 2 * ny + i] = eunit * lo;
                c->spec[(size_t)k * nf + 2 * ny + nx + i] = eunit * hi;
            }
        }
#undef AF
    }
    if (p->accept) { /* A4 subcycled per cell (Sec. 2.1 step 2, acceptance rule) */
        double *em = calloc(nc, sizeof(double)), *ab = calloc(nc, sizeof(double));
#pragma omp parallel for schedule(static)
        for (long long idl = 0; idl < (long long)nc; ++idl) {
            const size_t id = (size_t)idl;
            const int n = o_step2_subcycle(c, id, nc, dt, p->lum[id], 0, Jo, Hxo, Hyo, ax, ay, em, ab);
            if (c->nsub) c->nsub[id] = n;
        }
        for (size_t id = 0; id < nc; ++id) {
            o_kadd(&s_em, em[id]);
            o_kadd(&s_ab, ab[id]);
        }
        free(em);
        free(ab);
    }
    /* A5: f = 4 pi / (c ct dt) sum_k dnu_k (H' - H'') */
    const double fcoef = (4.0 * O_PI) / ((O_C * p->c_tilde) * dt);
    for (size_t id = 0; id < nc; ++id) {
        fx[id] = fcoef * ax[id];
        fy[id] = fcoef * ay[id];
    }

    /* A6: frequency step per cell, in place on (Jo, Hxo, Hyo) */
    if (!p->gray && p->freq_step) {
        double *nbc = malloc(nb * sizeof(double));
        for (int k = 0; k < nb; ++k) nbc[k] = c->nubar[k] / O_C;
#pragma omp parallel
        {
            double *scr = malloc((size_t)6 * nb * sizeof(double));
            double *Jin = malloc(nb * sizeof(double)), *Jn = malloc(nb * sizeof(double));
            double *DdU = malloc(nb * sizeof(double));
            double *Hcell = malloc(nb * sizeof(double)), *Rcell = malloc(nb * sizeof(double));
#pragma omp for schedule(static)
            for (long long idl = 0; idl < (long long)nc; ++idl) {
                size_t id = (size_t)idl;
                if (!(c->alpha[id] > 0.0)) {
                    for (int k = 0; k < nb; ++k) {
                        size_t kid = (size_t)k * nc + id;
                        o_causal(Jo[kid], &Hxo[kid], &Hyo[kid]);
                    }
                    continue;
                }
                for (int k = 0; k < nb; ++k) {
                    size_t kid = (size_t)k * nc + id;
                    o_prim q = o_make_prim(Jo[kid], Hxo[kid], Hyo[kid]);
                    double fxc = q.fn, fyc = q.ft, f2 = fxc * fxc + fyc * fyc;
                    if (f2 > 1.0) {
                        double r = sqrt(f2);
                        fxc = fxc / r;
                        fyc = fyc / r;
                    }
                    double Dxx, Dxy, Dyy;
                    o_closure(fxc, fyc, &Dxx, &Dxy, &Dyy);
                    DdU[k] = (Dxx * c->gxx[id] + Dyy * c->gyy[id]) + Dxy * c->gsh[id];
                    Jin[k] = Jo[kid];
                }
                o_freq_of_cell(c, id, nc, nbc, DdU, cdt, Jin, Jn, scr, Hcell, Rcell);
                for (int k = 0; k < nb; ++k) {
                    size_t kid = (size_t)k * nc + id;
                    double ratio = (Jin[k] > 0.0) ? Jn[k] / Jin[k] : 0.0;
                    Jo[kid] = Jn[k];
                    Hxo[kid] = ratio * Hxo[kid];
                    Hyo[kid] = ratio * Hyo[kid];
                    o_causal(Jo[kid], &Hxo[kid], &Hyo[kid]);
                }
            }
            free(scr); free(Jin); free(Jn); free(DdU); free(Hcell); free(Rcell);
        }
        free(nbc);
    }

    /* A7: diagnostics */
    d.e_after = o_energy(c, Jo);
    d.emitted = eunit * o_kval(&s_em);
    d.absorbed = eunit * o_kval(&s_ab);
    d.outflow = eunit * o_kval(&s_out);
    d.work = eunit * o_kval(&s_wk);
    d.residual = (d.e_after - d.e_before) - (((d.emitted - d.absorbed) - d.outflow) - d.work);
    double maxf = 0.0, nbad = 0.0;
    for (int k = 0; k < nb; ++k)
        for (size_t id = 0; id < nc; ++id) {
            size_t kid = (size_t)k * nc + id;
            double hn = sqrt(Hxo[kid] * Hxo[kid] + Hyo[kid] * Hyo[kid]);
            if (Jo[kid] > 0.0) {
                double f = hn / Jo[kid];
                if (f > maxf) maxf = f;
            }
            if (hn > Jo[kid] * (1.0 + 1e-12) && hn > 0.0) nbad += 1.0;
        }
    d.max_f = maxf;
    d.n_unrealisable = nbad;
    o_ksum fa = {0, 0}, fr = {0, 0};
    double cx = 0.5 * nx * dx, cy = 0.5 * ny * dx;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t id = (size_t)j * nx + i;
            double x = (i + 0.5) * dx - cx, y = (j + 0.5) * dx - cy, r = sqrt(x * x + y * y);
            o_kadd(&fa, sqrt(fx[id] * fx[id] + fy[id] * fy[id]) * V);
            if (r > 0.0) o_kadd(&fr, ((fx[id] * x + fy[id] * y) / r) * V);
        }
    d.force_abs = o_kval(&fa);
    d.force_radial = o_kval(&fr);
    if (dg) *dg = d;
    free(FJx); free(FHxx); free(FHyx); free(FJy); free(FHxy); free(FHyy); free(Wk); free(ax); free(ay);
    free(act);
    return 0;
}


/* ======================================================================
 * One substep in axisymmetric cylindrical geometry (R = x index, Z = y
 * index): finite volumes per radian, R faces of area R dZ, Z faces of area
 * (R+^2 - R-^2)/2, the hoop-stress source +K_phiphi <1/R> in the H_R
 * equation (the R component of div K in cylindrical coordinates), the
 * D_phiphi <u_R/R> parts of the work term and of D:grad(u) in step 3 (App. A),
 * mirrored ghosts at R = 0 and Z = 0 (H_R and u_R flip across the axis, H_Z
 * and u_Z across the midplane), outflow ghosts outside.
 * ====================================================================== */
int lym1o_substep_cyl(const lym1o_ctx *c, double dt, const double *J, const double *Hx,
                      const double *Hy, double *Jo, double *Hxo, double *Hyo, double *fx,
                      double *fy, lym1o_diag *dg)
{
    const lym1o_problem *p = &c->p;
    const int nx = p->nx, ny = p->ny, nb = c->nb;
    const size_t nc = (size_t)nx * ny;
    const double dx = p->dx, half_dx = 0.5 * dx, cdt = p->c_tilde * dt;
    lym1o_diag d;
    memset(&d, 0, sizeof d);
    o_ksum s_e0 = {0, 0}, s_e1 = {0, 0}, s_em = {0, 0}, s_ab = {0, 0}, s_out = {0, 0}, s_wk = {0, 0};
    for (int k = 0; k < nb; ++k)
        for (size_t id = 0; id < nc; ++id)
            o_kadd(&s_e0, c->V2pi[id % nx] * (c->dnu[k] * J[(size_t)k * nc + id]));
    double *FJx = malloc((size_t)(nx + 1) * ny * sizeof(double));
    double *FHxx = malloc((size_t)(nx + 1) * ny * sizeof(double));
    double *FHyx = malloc((size_t)(nx + 1) * ny * sizeof(double));
    double *FJy = malloc((size_t)nx * (ny + 1) * sizeof(double));
    double *FHxy = malloc((size_t)nx * (ny + 1) * sizeof(double));
    double *FHyy = malloc((size_t)nx * (ny + 1) * sizeof(double));
    double *Wk = malloc(nc * sizeof(double));
    double *ax = calloc(nc, sizeof(double)), *ay = calloc(nc, sizeof(double));
    unsigned char *act = o_active_bins(c, J);

    for (int k = 0; k < nb; ++k) {
        const double *Jk = J + (size_t)k * nc, *Hxk = Hx + (size_t)k * nc, *Hyk = Hy + (size_t)k * nc;
#define AFC(id) (p->band_aF ? BND(band_aF, k, id) : c->alpha[id] * HAV(k, id) + p->rho_d[id] * p->kappa_F)
        const int on = !act || act[k]; /* pruned bins: no step 1 */
        if (!on) {
            o_zero(FJx, (size_t)(nx + 1) * ny);
            o_zero(FHxx, (size_t)(nx + 1) * ny);
            o_zero(FHyx, (size_t)(nx + 1) * ny);
            o_zero(FJy, (size_t)nx * (ny + 1));
            o_zero(FHxy, (size_t)nx * (ny + 1));
            o_zero(FHyy, (size_t)nx * (ny + 1));
        } else {
        /* R faces: face i between cells i-1 and i */
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                int fl[4];
                int ii[4];
                for (int m = 0; m < 4; ++m) ii[m] = o_mir(i - 2 + m, nx, &fl[m]);
                o_prim q[4];
                double ur[2];
                for (int m = 0; m < 4; ++m) {
                    size_t id = (size_t)j * nx + ii[m];
                    double sg = fl[m] ? -1.0 : 1.0;
                    q[m] = o_vac(i - 2 + m, nx, 0, p->bc[1]) ? o_make_prim(0.0, 0.0, 0.0)
                                                             : o_make_prim(Jk[id], Hxk[id] * sg, Hyk[id]);
                    if (m == 1 || m == 2) ur[m - 1] = p->ux[id] * sg;
                }
                size_t i0 = (size_t)j * nx + ii[1], i1 = (size_t)j * nx + ii[2];
                size_t f = (size_t)j * (nx + 1) + i;
                o_face(q[0], q[1], q[2], q[3], AFC(i0), AFC(i1), ur[0], ur[1], c->dlL[i], c->dlR[i],
                       &FJx[f], &FHxx[f], &FHyx[f]);
            }
        /* Z faces: face j between rows j-1 and j */
#pragma omp parallel for schedule(static)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int fl[4];
                int jj[4];
                for (int m = 0; m < 4; ++m) jj[m] = o_mir(j - 2 + m, ny, &fl[m]);
                o_prim q[4];
                double uz[2];
                for (int m = 0; m < 4; ++m) {
                    size_t id = (size_t)jj[m] * nx + i;
                    double sg = fl[m] ? -1.0 : 1.0;
                    q[m] = o_vac(j - 2 + m, ny, 0, p->bc[3]) ? o_make_prim(0.0, 0.0, 0.0)
                                                             : o_make_prim(Jk[id], Hyk[id] * sg, Hxk[id]);
                    if (m == 1 || m == 2) uz[m - 1] = p->uy[id] * sg;
                }
                size_t i0 = (size_t)jj[1] * nx + i, i1 = (size_t)jj[2] * nx + i;
                size_t f = (size_t)j * nx + i;
                o_face(q[0], q[1], q[2], q[3], AFC(i0), AFC(i1), uz[0], uz[1], half_dx, half_dx,
                       &FJy[f], &FHyy[f], &FHxy[f]);
            }
        }
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t id = (size_t)j * nx + i, kid = (size_t)k * nc + id;
                o_prim q = o_make_prim(Jk[id], Hxk[id], Hyk[id]);
                double fxc = q.fn, fyc = q.ft, f2 = fxc * fxc + fyc * fyc;
                if (f2 > 1.0) {
                    double r = sqrt(f2);
                    fxc = fxc / r;
                    fyc = fyc / r;
                }
                double Dxx, Dxy, Dyy;
                o_closure(fxc, fyc, &Dxx, &Dxy, &Dyy);
                double f2c = fxc * fxc + fyc * fyc;
                double chi = (3.0 + 4.0 * f2c) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f2c));
                double Dpp = (1.0 - chi) / 2.0;
                double W = (((Dxx * Jk[id]) * c->gxx[id] + (Dyy * Jk[id]) * c->gyy[id]) +
                            (Dxy * Jk[id]) * c->gsh[id]) +
                           (Dpp * Jk[id]) * c->gphi[id];
                if (!on) W = 0.0;
                Wk[id] = W;
                size_t fxl = (size_t)j * (nx + 1) + i, fyl = (size_t)j * nx + i;
                double divJ = ((c->AR[i + 1] * FJx[fxl + 1] - c->AR[i] * FJx[fxl]) +
                               c->AZ[i] * (FJy[fyl + nx] - FJy[fyl])) / c->Vol[i];
                double divHx = ((c->AR[i + 1] * FHxx[fxl + 1] - c->AR[i] * FHxx[fxl]) +
                                c->AZ[i] * (FHxy[fyl + nx] - FHxy[fyl])) / c->Vol[i] -
                               (Dpp * Jk[id]) * c->invR[i];
                if (!on) divHx = 0.0;
                double divHy = ((c->AR[i + 1] * FHyx[fxl + 1] - c->AR[i] * FHyx[fxl]) +
                                c->AZ[i] * (FHyy[fyl + nx] - FHyy[fyl])) / c->Vol[i];
                double J1 = Jk[id] - cdt * (divJ + W / O_C);
                double Hx1 = Hxk[id] - cdt * divHx;
                double Hy1 = Hyk[id] - cdt * divHy;
                double aH = c->alpha[id] * HAV(k, id);
                double kap = p->rho_d[id] * p->kappa_abs + p->p_d[id] * aH;
                double aF = aH + p->rho_d[id] * p->kappa_F;
                double js = (p->lum[id] / c->V2pi[i]) * GEMC(k, id);
                if (p->band_aF) {
                    kap = BND(band_kap, k, id);
                    aF = BND(band_aF, k, id);
                    js = BND(band_j, k, id);
                }
                if (p->accept) { /* step 2 is subcycled per cell after the bin loop */
                    Jo[kid] = J1;
                    Hxo[kid] = Hx1;
                    Hyo[kid] = Hy1;
                    continue;
                }
                double J2 = (J1 + cdt * js) / (1.0 + cdt * kap);
                double Hx2 = Hx1 / (1.0 + cdt * aF);
                double Hy2 = Hy1 / (1.0 + cdt * aF);
                Jo[kid] = J2;
                Hxo[kid] = Hx2;
                Hyo[kid] = Hy2;
                ax[id] = ax[id] + c->dnu[k] * (Hx1 - Hx2);
                ay[id] = ay[id] + c->dnu[k] * (Hy1 - Hy2);
            }
        for (size_t id = 0; id < nc; ++id) {
            size_t kid = (size_t)k * nc + id;
            int i = (int)(id % nx);
            double aH = c->alpha[id] * HAV(k, id);
            double kap = p->rho_d[id] * p->kappa_abs + p->p_d[id] * aH;
            double js = (p->lum[id] / c->V2pi[i]) * GEMC(k, id);
            if (p->band_aF) {
                kap = BND(band_kap, k, id);
                js = BND(band_j, k, id);
            }
            if (!p->accept) {
                o_kadd(&s_em, c->V2pi[i] * (c->dnu[k] * (cdt * js)));
                o_kadd(&s_ab, c->V2pi[i] * (c->dnu[k] * (cdt * (kap * Jo[kid]))));
            }
            o_kadd(&s_wk, c->V2pi[i] * (c->dnu[k] * (cdt * (Wk[id] / O_C))));
        }
        /* outflow through the outer R and Z faces (the axis and midplane are mirrors) */
        const int nf = nx + ny;
        for (int j = 0; j < ny; ++j) {
            double o = (2.0 * O_PI) * (c->AR[nx] * (c->dnu[k] * (cdt * FJx[(size_t)j * (nx + 1) + nx])));
            o_kadd(&s_out, o);
            if (c->spec) c->spec[(size_t)k * nf + j] = ((4.0 * O_PI) / O_C) * o;
        }
        for (int i = 0; i < nx; ++i) {
            double o = (2.0 * O_PI) * (c->AZ[i] * (c->dnu[k] * (cdt * FJy[(size_t)ny * nx + i])));
            o_kadd(&s_out, o);
            if (c->spec) c->spec[(size_t)k * nf + ny + i] = ((4.0 * O_PI) / O_C) * o;
        }
#undef AFC
    }
    if (p->accept) { /* A4 subcycled per cell (Sec. 2.1 step 2, acceptance rule) */
        double *em = calloc(nc, sizeof(double)), *ab = calloc(nc, sizeof(double));
#pragma omp parallel for schedule(static)
        for (long long idl = 0; idl < (long long)nc; ++idl) {
            const size_t id = (size_t)idl;
            const int i = (int)(id % nx);
            const int n = o_step2_subcycle(c, id, nc, dt, p->lum[id] / c->V2pi[i], 1, Jo, Hxo, Hyo,
                                           ax, ay, em, ab);
            if (c->nsub) c->nsub[id] = n;
        }
        for (size_t id = 0; id < nc; ++id) {
            o_kadd(&s_em, c->V2pi[id % nx] * em[id]);
            o_kadd(&s_ab, c->V2pi[id % nx] * ab[id]);
        }
        free(em);
        free(ab);
    }
    const double fcoef = (4.0 * O_PI) / ((O_C * p->c_tilde) * dt);
    for (size_t id = 0; id < nc; ++id) {
        fx[id] = fcoef * ax[id];
        fy[id] = fcoef * ay[id];
    }
    if (!p->gray && p->freq_step) {
        double *nbc = malloc(nb * sizeof(double));
        for (int k = 0; k < nb; ++k) nbc[k] = c->nubar[k] / O_C;
#pragma omp parallel
        {
            double *scr = malloc((size_t)6 * nb * sizeof(double));
            double *Jin = malloc(nb * sizeof(double)), *Jn = malloc(nb * sizeof(double));
            double *DdU = malloc(nb * sizeof(double));
            double *Hcell = malloc(nb * sizeof(double)), *Rcell = malloc(nb * sizeof(double));
#pragma omp for schedule(static)
            for (long long idl = 0; idl < (long long)nc; ++idl) {
                size_t id = (size_t)idl;
                if (!(c->alpha[id] > 0.0)) {
                    for (int k = 0; k < nb; ++k) {
                        size_t kid = (size_t)k * nc + id;
                        o_causal(Jo[kid], &Hxo[kid], &Hyo[kid]);
                    }
                    continue;
                }
                for (int k = 0; k < nb; ++k) {
                    size_t kid = (size_t)k * nc + id;
                    o_prim q = o_make_prim(Jo[kid], Hxo[kid], Hyo[kid]);
                    double fxc = q.fn, fyc = q.ft, f2 = fxc * fxc + fyc * fyc;
                    if (f2 > 1.0) {
                        double r = sqrt(f2);
                        fxc = fxc / r;
                        fyc = fyc / r;
                    }
                    double Dxx, Dxy, Dyy;
                    o_closure(fxc, fyc, &Dxx, &Dxy, &Dyy);
                    double f2c = fxc * fxc + fyc * fyc;
                    double chi = (3.0 + 4.0 * f2c) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f2c));
                    double Dpp = (1.0 - chi) / 2.0;
                    DdU[k] = ((Dxx * c->gxx[id] + Dyy * c->gyy[id]) + Dxy * c->gsh[id]) +
                             Dpp * c->gphi[id];
                    Jin[k] = Jo[kid];
                }
                o_freq_of_cell(c, id, nc, nbc, DdU, cdt, Jin, Jn, scr, Hcell, Rcell);
                for (int k = 0; k < nb; ++k) {
                    size_t kid = (size_t)k * nc + id;
                    double ratio = (Jin[k] > 0.0) ? Jn[k] / Jin[k] : 0.0;
                    Jo[kid] = Jn[k];
                    Hxo[kid] = ratio * Hxo[kid];
                    Hyo[kid] = ratio * Hyo[kid];
                    o_causal(Jo[kid], &Hxo[kid], &Hyo[kid]);
                }
            }
            free(scr); free(Jin); free(Jn); free(DdU); free(Hcell); free(Rcell);
        }
        free(nbc);
    }
    for (int k = 0; k < nb; ++k)
        for (size_t id = 0; id < nc; ++id)
            o_kadd(&s_e1, c->V2pi[id % nx] * (c->dnu[k] * Jo[(size_t)k * nc + id]));
    const double eu = (4.0 * O_PI) / O_C;
    d.e_before = eu * o_kval(&s_e0);
    d.e_after = eu * o_kval(&s_e1);
    d.emitted = eu * o_kval(&s_em);
    d.absorbed = eu * o_kval(&s_ab);
    d.outflow = eu * o_kval(&s_out);
    d.work = eu * o_kval(&s_wk);
    d.residual = (d.e_after - d.e_before) - (((d.emitted - d.absorbed) - d.outflow) - d.work);
    double maxf = 0.0, nbad = 0.0;
    for (int k = 0; k < nb; ++k)
        for (size_t id = 0; id < nc; ++id) {
            size_t kid = (size_t)k * nc + id;
            double hn = sqrt(Hxo[kid] * Hxo[kid] + Hyo[kid] * Hyo[kid]);
            if (Jo[kid] > 0.0 && hn / Jo[kid] > maxf) maxf = hn / Jo[kid];
            if (hn > Jo[kid] * (1.0 + 1e-12) && hn > 0.0) nbad += 1.0;
        }
    d.max_f = maxf;
    d.n_unrealisable = nbad;
    o_ksum fa = {0, 0}, fr = {0, 0};
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t id = (size_t)j * nx + i;
            double R = (i + 0.5) * dx, Z = (j + 0.5) * dx, r = sqrt(R * R + Z * Z);
            o_kadd(&fa, sqrt(fx[id] * fx[id] + fy[id] * fy[id]) * c->V2pi[i]);
            o_kadd(&fr, ((fx[id] * R + fy[id] * Z) / r) * c->V2pi[i]);
        }
    d.force_abs = o_kval(&fa);
    d.force_radial = o_kval(&fr);
    if (dg) *dg = d;
    free(FJx); free(FHxx); free(FHyx); free(FJy); free(FHxy); free(FHyy); free(Wk); free(ax); free(ay);
    free(act);
    return 0;
}

/* ======================================================================
 * Reduced speed of light.  lym1o_set_ctilde sets c_tilde and the RT time
 * step (Sec. 2.1, CFL condition).  lym1o_dynamic_ctilde applies the dynamic
 * choice of Sec. 2.1 (the dynamic-RSL equation and its f_abs factor):
 *   c_dyn = eps_RSL max_cells { max[1, (a_v tau_0)^(1/3) f_abs] max[|u|, c_s] },
 *   f_abs = 1 / (1 + (a_v tau_0)^(1/3) tau_c + 0.6 p_d tau_0),
 * with tau_0 = alpha dx the cell's line-centre optical depth (square cells)
 * and tau_c = rho_d kappa_abs dx its continuum absorption depth; then
 * c_tilde = min[max(c_min, c_dyn), c], moved by at most -25 % or x4 from the
 * current value.  cs: per-cell sound speed (cm/s), or NULL for that of
 * neutral atomic gas at the cell's temperature (gamma = 5/3, mu = 1.22).
 * Returns the new c_tilde.
 * ====================================================================== */
void lym1o_set_ctilde(lym1o_ctx *c, double ct)
{
    c->p.c_tilde = ct;
    c->dt_cfl = (c->p.cfl / 2.0) * (c->p.dx / (ct + c->umax));
}

double lym1o_dynamic_ctilde(lym1o_ctx *c, const double *cs, double eps_rsl, double ct_min)
{
    const lym1o_problem *p = &c->p;
    const size_t nc = (size_t)p->nx * p->ny;
    double m = 0.0;
    for (size_t id = 0; id < nc; ++id) {
        const double T = p->temp ? p->temp[id] : p->T;
        double lc[3];
        lym1o_line(T, lc);
        const double tau0 = c->alpha[id] * p->dx;
        const double tauc = (p->rho_d[id] * p->kappa_abs) * p->dx;
        const double X = cbrt(lc[1] * tau0);
        const double fabs_ = 1.0 / ((1.0 + X * tauc) + (0.6 * p->p_d[id]) * tau0);
        const double u = sqrt(p->ux[id] * p->ux[id] + p->uy[id] * p->uy[id]);
        const double s = cs ? cs[id] : sqrt(((5.0 / 3.0) * (O_KB * T)) / (1.22 * O_MH));
        const double term = fmax(1.0, X * fabs_) * fmax(u, s);
        if (term > m) m = term;
    }
    double ct = fmin(fmax(ct_min, eps_rsl * m), O_C);
    const double prev = p->c_tilde;
    ct = fmin(fmax(ct, 0.75 * prev), 4.0 * prev);
    lym1o_set_ctilde(c, ct);
    return ct;
}

/* emergent spectrum output of the following substeps (NULL: off); buf holds
 * nb x (2 (nx + ny)) doubles for geometry 0, nb x (nx + ny) for geometry 1 */
void lym1o_set_spectrum(lym1o_ctx *c, double *buf) { c->spec = buf; }
void lym1o_set_subcycle_out(lym1o_ctx *c, int *buf) { c->nsub = buf; }

void lym1o_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int lym1o_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
