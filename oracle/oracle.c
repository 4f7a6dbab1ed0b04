/*
 * FP64 CPU oracle for list-mode MLEM reconstruction in the two-strip detector
 * (Bialas et al., "GPU accelerated image reconstruction in a two-strip J-PET
 * tomograph", arXiv:1502.07478).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, double-precision
 * statement of what the reconstruction computes.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header or constant table with the CUDA library.
 *
 * Sections of the paper followed here:
 *   Eq. 1 (Sec. 2)      measurement model of delta_l
 *   Eq. 2 (Sec. 2)      direct reconstruction of (y, z, tan theta) from one event
 *   Eq. iter            one list-mode MLEM update, with the sensitivity s
 *   Eq. iter-p          the same update written for rho' = s rho
 *   Eq. s-yz            sensitivity of a pixel from the strip geometry
 *   Eq. kernel (Sec. 3) Laplace-approximated event kernel P(e|i) with o, a, b, C^-1
 *   Sec. 3, App. B      3-sigma ellipse window and its bounding box
 *   Sec. 4, Listing 1   the per-event two-pass structure: cache P over the
 *                       window while summing the denominator, then scatter
 *   Sec. 4.1            OpenMP over events, each thread with its own copy of
 *                       the new image, summed at the end of the iteration
 *
 * Readings of passages that are garbled or silent (each also listed in the
 * design notes):
 *   R1 Eq. 2: the second forms of y and z lack a square and carry a wrong factor;
 *      the first forms are used.
 *   R2 Strip at y = +R is the upper strip; z_u = z + (R - y) tan(theta),
 *      z_d = z - (R + y) tan(theta), delta_l = -2 y / cos(theta); "cos^-1" in the
 *      definitions of o, a, b means sec, not arccos.
 *   R3 a_3: differentiating e_3(theta) = -2 y sec(theta) gives
 *      a_3 = -2 y tan sec; the printed a_3 lacks the 2.  The derived form is the
 *      default; the a3_printed flag selects the printed one.
 *   R4 Prefactor: det^(1/2) is taken of C^-1 and the uniform angle density
 *      1/pi is included, so P = det^(1/2)(C^-1) / (2 pi^2 sqrt(Q)) exp(...).
 *      A constant factor cancels in Eq. iter.
 *   R5 Q = aC^-1a + 2 oC^-1b <= 0 gives P = 0 (counted).
 *   R6 Window: pixel i belongs to event j iff b C^-1 b <= cut^2 at the pixel
 *      centre.  The bounding box only bounds the loop; it is padded by one pixel
 *      and clipped to the grid.
 *   R7 App. B's ellipse equation lacks a factor 2 on the cross term; the
 *      bounding-box half-extents used are h_y = cut sigma_dl cos/2 and
 *      h_z = cut sqrt(sigma_z^2/2 + sigma_dl^2 sin^2/4).
 *   R8 Listing 1's rho[l] in the scatter is rho[i]; the listing is Eq. iter-p.
 *   R9 Sensitivity at pixel centres, clamped to >= 0.
 *   R10 Events with D_j = 0 are skipped and counted; then sum_l s_l rho_l = N_used.
 *   R15 Sec. 3 notes that the z resolution degrades by about 10% from the centre
 *      of the strips to their ends, without a functional form.  With kappa_z != 0
 *      an event reconstructed at z~ uses sigma_z (1 + kappa_z min(1, (2 z~/L)^2))
 *      in its kernel, window and box (kappa_z = 0.1: 10% at the ends); the
 *      gradient is taken with respect to the base sigma_z.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
    double R;          /* half of the strip separation: strips at y = +R, -R (mm) */
    double L;          /* strip length (mm) */
    int32_t ny, nz;    /* image grid: ny rows (y), nz columns (z, contiguous) */
    double dy, dz;     /* pixel pitch (mm) */
    double sigma_z;    /* kernel resolution of z_u and z_d (mm) */
    double sigma_dl;   /* kernel resolution of delta_l (mm) */
    double gamma;      /* off-diagonal term of C^-1 (Sec. 3); 0 = diagonal */
    double cut;        /* window radius in sigma units (3) */
    double wsigma_z;   /* window sigmas; 0 = same as the kernel's (a frozen  */
    double wsigma_dl;  /*   window for finite differences uses the base values) */
    double pscale;     /* extra constant factor on P (1); tests that it cancels */
    int32_t a3_printed;/* 1 = use the printed a_3 (reading R3) */
    int32_t form_p;    /* 1 = iterate Eq. iter-p on rho' (no s); 0 = Eq. iter */
    int32_t n_threads; /* OpenMP threads; <= 0 = library default */
    int32_t pad_;
    double kappa_z;    /* z dependence of sigma_z (reading R15); 0 = constant */
} orc_params;

typedef struct {
    int64_t n_used;     /* events with D_j > 0 */
    int64_t n_empty;    /* events with D_j = 0 (skipped) */
    int64_t n_window;   /* sum over events of in-window pixels (pixel evaluations) */
    int64_t n_qbad;     /* in-window pixels with Q <= 0 (P set to 0) */
    double sum_s_rho;   /* sum_l s_l rho_l after the last update */
} orc_stats;

/* ---------------------------------------------------------------- geometry */

/* Eq. 2, first forms: tan(theta) = (z_u - z_d)/(2R), y = -dl/2 / sqrt(1+tan^2),
 * z = (z_u + z_d + 2 y tan(theta))/2. */
void orc_direct(const orc_params* p, double zu, double zd, double dl,
                double* y, double* z, double* tan_theta)
{
    double t = (zu - zd) / (2.0 * p->R);
    double yy = -0.5 * dl / sqrt(1.0 + t * t);
    *tan_theta = t;
    *y = yy;
    *z = 0.5 * (zu + zd + 2.0 * yy * t);
}

/* Eq. 1: the path-length difference of an emission at (y, z) seen at (z_u, z_d). */
double orc_delta_l(const orc_params* p, double y, double z, double zu, double zd)
{
    double R = p->R;
    return sqrt((R - y) * (R - y) + (zu - z) * (zu - z))
         - sqrt((R + y) * (R + y) + (zd - z) * (zd - z));
}

/* Eq. s-yz: fraction of emission angles from (y, z) whose line hits both strips. */
double orc_sensitivity_at(const orc_params* p, double y, double z)
{
    double R = p->R, hl = 0.5 * p->L;
    if (!(fabs(y) < R)) return 0.0;
    double tmax = fmin((hl - z) / (R - y), (hl + z) / (R + y));
    double tmin = fmax(-(hl + z) / (R - y), (-hl + z) / (R + y));
    double s = (atan(tmax) - atan(tmin)) / ORC_PI;
    return s > 0.0 ? s : 0.0;
}

static double pix_y(const orc_params* p, int iy) { return -p->R + (iy + 0.5) * p->dy; }
static double pix_z(const orc_params* p, int iz) { return -0.5 * p->L + (iz + 0.5) * p->dz; }

void orc_sensitivity(const orc_params* p, double* s)
{
    for (int iy = 0; iy < p->ny; ++iy)
        for (int iz = 0; iz < p->nz; ++iz)
            s[(int64_t)iy * p->nz + iz] = orc_sensitivity_at(p, pix_y(p, iy), pix_z(p, iz));
}

/* ------------------------------------------------------- correlation matrix */

/* Reading R15: the factor on sigma_z for an event reconstructed at z~ = ez. */
static double zfactor(const orc_params* p, double ez)
{
    double s = 2.0 * ez / p->L;
    s = s * s;
    if (s > 1.0) s = 1.0;
    return 1.0 + p->kappa_z * s;
}

/* C^-1 of Sec. 3 for the given sigmas (general form with the cross term gamma). */
static void cinv_matrix(double sz, double sdl, double g, double C[3][3])
{
    double iz = 1.0 / (sz * sz), il = 1.0 / (sdl * sdl);
    C[0][0] = iz;  C[0][1] = 0.0; C[0][2] = g;
    C[1][0] = 0.0; C[1][1] = iz;  C[1][2] = -g;
    C[2][0] = g;   C[2][1] = -g;  C[2][2] = il;
}

static double quad(const double u[3], double C[3][3], const double v[3])
{
    double acc = 0.0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            acc += u[r] * C[r][c] * v[c];
    return acc;
}

static double det3(double C[3][3])
{
    return C[0][0] * (C[1][1] * C[2][2] - C[1][2] * C[2][1])
         - C[0][1] * (C[1][0] * C[2][2] - C[1][2] * C[2][0])
         + C[0][2] * (C[1][0] * C[2][1] - C[1][1] * C[2][0]);
}

static void inv3(double C[3][3], double I[3][3])
{
    double d = det3(C);
    I[0][0] = (C[1][1] * C[2][2] - C[1][2] * C[2][1]) / d;
    I[0][1] = (C[0][2] * C[2][1] - C[0][1] * C[2][2]) / d;
    I[0][2] = (C[0][1] * C[1][2] - C[0][2] * C[1][1]) / d;
    I[1][0] = (C[1][2] * C[2][0] - C[1][0] * C[2][2]) / d;
    I[1][1] = (C[0][0] * C[2][2] - C[0][2] * C[2][0]) / d;
    I[1][2] = (C[0][2] * C[1][0] - C[0][0] * C[1][2]) / d;
    I[2][0] = (C[1][0] * C[2][1] - C[1][1] * C[2][0]) / d;
    I[2][1] = (C[0][1] * C[2][0] - C[0][0] * C[2][1]) / d;
    I[2][2] = (C[0][0] * C[1][1] - C[0][1] * C[1][0]) / d;
}

/* ---------------------------------------------------------------- kernel P */

/* The vectors o, a, b of Sec. 3 for an event reconstructed at (ey, ez, tan et)
 * and a pixel centred at (py, pz).  Written out from their printed definitions
 * (with reading R3 for a_3). */
static void oab_vectors(const orc_params* p, double ey, double ez, double t,
                        double py, double pz, double o[3], double a[3], double b[3])
{
    double R = p->R;
    double sec = sqrt(1.0 + t * t);       /* 1/cos(theta~) */
    double sec2 = sec * sec;
    double dy = py - ey, dz = pz - ez;     /* Delta y, Delta z */
    o[0] = -(dy + ey - R) * t * sec2;
    o[1] = -(dy + ey + R) * t * sec2;
    o[2] = -(dy + ey) * sec * (1.0 + 2.0 * t * t);
    a[0] = -(dy + ey - R) * sec2;
    a[1] = -(dy + ey + R) * sec2;
    a[2] = (p->a3_printed ? -1.0 : -2.0) * (dy + ey) * sec * t;
    b[0] = dz - dy * t;
    b[1] = dz - dy * t;
    b[2] = -2.0 * dy * sec;
}

/* b C^-1 b with the window sigmas: the 3-sigma ellipse test quantity (R6). */
static double window_bq(const orc_params* p, double ey, double ez, double t,
                        double py, double pz)
{
    double C[3][3], o[3], a[3], b[3];
    double wz = (p->wsigma_z > 0 ? p->wsigma_z : p->sigma_z) * zfactor(p, ez);
    double wl = p->wsigma_dl > 0 ? p->wsigma_dl : p->sigma_dl;
    cinv_matrix(wz, wl, p->gamma, C);
    oab_vectors(p, ey, ez, t, py, pz, o, a, b);
    return quad(b, C, b);
}

/* Eq. kernel (reading R4, R5).  Returns P; *qbad = 1 when Q <= 0. */
static double kernel_value(const orc_params* p, double ey, double ez, double t,
                           double py, double pz, int* qbad)
{
    double C[3][3], o[3], a[3], b[3];
    cinv_matrix(p->sigma_z * zfactor(p, ez), p->sigma_dl, p->gamma, C);
    oab_vectors(p, ey, ez, t, py, pz, o, a, b);
    double aCa = quad(a, C, a), oCb = quad(o, C, b), bCb = quad(b, C, b), aCb = quad(a, C, b);
    double Q = aCa + 2.0 * oCb;
    if (qbad) *qbad = 0;
    if (!(Q > 0.0)) {
        if (qbad) *qbad = 1;
        return 0.0;
    }
    double pref = sqrt(det3(C)) / (2.0 * ORC_PI * ORC_PI * sqrt(Q));
    return p->pscale * pref * exp(-0.5 * (bCb - aCb * aCb / Q));
}

/* d log P / d sigma_z and d log P / d sigma_dl at fixed window (reading R4),
 * from log P = 1/2 log det C^-1 - 1/2 log Q - 1/2 bC^-1b + 1/2 (aC^-1b)^2/Q + const.
 * sigma_z is the base value: the event's own sigma_z is f sigma_z (reading R15),
 * so d(C^-1)_zz / d sigma_z = -2 f / (f sigma_z)^3. */
static void kernel_dlog(const orc_params* p, double ey, double ez, double t,
                        double py, double pz, double dlog[2])
{
    double C[3][3], Ci[3][3], o[3], a[3], b[3];   /* C holds C^-1 */
    double f = zfactor(p, ez);
    cinv_matrix(p->sigma_z * f, p->sigma_dl, p->gamma, C);
    inv3(C, Ci);
    oab_vectors(p, ey, ez, t, py, pz, o, a, b);
    double aCa = quad(a, C, a), oCb = quad(o, C, b), bCb = quad(b, C, b), aCb = quad(a, C, b);
    double Q = aCa + 2.0 * oCb;
    (void)bCb;
    double sz = p->sigma_z * f, sl = p->sigma_dl;
    for (int k = 0; k < 2; ++k) {
        double dC[3][3];
        memset(dC, 0, sizeof dC);
        if (k == 0) { dC[0][0] = dC[1][1] = -2.0 * f / (sz * sz * sz); }
        else        { dC[2][2] = -2.0 / (sl * sl * sl); }
        /* d log det(C^-1) = tr(C d(C^-1)); Ci holds C, the inverse of C^-1 */
        double tr = 0.0;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                tr += Ci[c][r] * dC[r][c];
        double dQ = quad(a, dC, a) + 2.0 * quad(o, dC, b);
        double dbb = quad(b, dC, b);
        double dab = quad(a, dC, b);
        dlog[k] = 0.5 * tr - 0.5 * dQ / Q - 0.5 * dbb + aCb * dab / Q
                - 0.5 * aCb * aCb * dQ / (Q * Q);
    }
}

double orc_kernel(const orc_params* p, double ey, double ez, double t,
                  double py, double pz, double* bq_out)
{
    if (bq_out) *bq_out = window_bq(p, ey, ez, t, py, pz);
    return kernel_value(p, ey, ez, t, py, pz, NULL);
}

/* Eq. kernel over arrays: P[k] and b C^-1 b [k] for event k at (ey, ez, t) and
 * pixel centre (py, pz); bq may be NULL. */
void orc_kernel_batch(const orc_params* p, int64_t n, const double* ey, const double* ez,
                      const double* t, const double* py, const double* pz,
                      double* P, double* bq)
{
    for (int64_t k = 0; k < n; ++k) {
        if (bq) bq[k] = window_bq(p, ey[k], ez[k], t[k], py[k], pz[k]);
        P[k] = kernel_value(p, ey[k], ez[k], t[k], py[k], pz[k], NULL);
    }
}

void orc_kernel_dlog(const orc_params* p, double ey, double ez, double t,
                     double py, double pz, double* dlog2)
{
    kernel_dlog(p, ey, ez, t, py, pz, dlog2);
}

/* App. B (reading R7): half-extents of the bounding box of the cut ellipse of an
 * event at z~ = ez (which sets its sigma_z, reading R15). */
void orc_bbox(const orc_params* p, double ez, double t, double* hy, double* hz)
{
    double wz = (p->wsigma_z > 0 ? p->wsigma_z : p->sigma_z) * zfactor(p, ez);
    double wl = p->wsigma_dl > 0 ? p->wsigma_dl : p->sigma_dl;
    double c2 = 1.0 / (1.0 + t * t), s2 = 1.0 - c2;
    *hy = p->cut * wl * sqrt(c2) / 2.0;
    *hz = p->cut * sqrt(wz * wz / 2.0 + wl * wl * s2 / 4.0);
}

/* ---------------------------------------------------------- per-event pass */

typedef struct {
    int64_t* idx;    /* cached in-window pixel indices (Listing 1's kernel cache) */
    double* P;       /* cached kernel values */
    int64_t cap;
} cache_t;

static void cache_reserve(cache_t* c, int64_t n)
{
    if (n <= c->cap) return;
    c->idx = (int64_t*)realloc(c->idx, (size_t)n * sizeof(int64_t));
    c->P = (double*)realloc(c->P, (size_t)n * sizeof(double));
    c->cap = n;
}

/* Pass 1 of Listing 1 for one event: loop over the (padded, clipped) bounding
 * box, keep pixels inside the ellipse, cache P.  Returns the number cached. */
static int64_t event_window(const orc_params* p, double zu, double zd, double dl,
                            cache_t* c, int64_t* qbad,
                            double* ey_o, double* ez_o, double* t_o)
{
    double ey, ez, t;
    orc_direct(p, zu, zd, dl, &ey, &ez, &t);
    *ey_o = ey; *ez_o = ez; *t_o = t;
    double hy, hz;
    orc_bbox(p, ez, t, &hy, &hz);
    double y0 = -p->R + 0.5 * p->dy, z0 = -0.5 * p->L + 0.5 * p->dz;
    double fy_lo = floor((ey - hy - y0) / p->dy) - 1, fy_hi = ceil((ey + hy - y0) / p->dy) + 1;
    double fz_lo = floor((ez - hz - z0) / p->dz) - 1, fz_hi = ceil((ez + hz - z0) / p->dz) + 1;
    if (fy_hi < 0 || fz_hi < 0 || fy_lo > p->ny - 1 || fz_lo > p->nz - 1) return 0;
    int iy_lo = fy_lo < 0 ? 0 : (int)fy_lo, iy_hi = fy_hi > p->ny - 1 ? p->ny - 1 : (int)fy_hi;
    int iz_lo = fz_lo < 0 ? 0 : (int)fz_lo, iz_hi = fz_hi > p->nz - 1 ? p->nz - 1 : (int)fz_hi;
    cache_reserve(c, (int64_t)(iy_hi - iy_lo + 1) * (iz_hi - iz_lo + 1));
    int64_t n = 0;
    double cut2 = p->cut * p->cut;
    for (int iy = iy_lo; iy <= iy_hi; ++iy) {
        double py = pix_y(p, iy);
        for (int iz = iz_lo; iz <= iz_hi; ++iz) {
            double pz = pix_z(p, iz);
            if (window_bq(p, ey, ez, t, py, pz) <= cut2) {
                int qb = 0;
                c->idx[n] = (int64_t)iy * p->nz + iz;
                c->P[n] = kernel_value(p, ey, ez, t, py, pz, &qb);
                *qbad += qb;
                ++n;
            }
        }
    }
    return n;
}

static int nthreads_of(const orc_params* p)
{
#ifdef _OPENMP
    return p->n_threads > 0 ? p->n_threads : omp_get_max_threads();
#else
    (void)p;
    return 1;
#endif
}

/* One or more MLEM iterations (Eq. iter, or Eq. iter-p when form_p = 1).
 * rho (ny*nz) is updated in place; s is the sensitivity (ignored for iter-p).
 * loglik (nullable, n_iter entries) receives the log-likelihood of the image
 * entering each iteration: sum_j log D_j - sum_i s_i rho_i. */
int orc_mlem(const orc_params* p, const double* zu, const double* zd, const double* dl,
             int64_t n, const double* s, double* rho, int n_iter,
             double* loglik, orc_stats* st)
{
    int64_t npix = (int64_t)p->ny * p->nz;
    int nt = nthreads_of(p);
    double* partial = (double*)calloc((size_t)nt * npix, sizeof(double));
    if (!partial) return -1;
    for (int it = 0; it < n_iter; ++it) {
        int64_t n_used = 0, n_empty = 0, n_window = 0, n_qbad = 0;
        double sum_log = 0.0;
        memset(partial, 0, (size_t)nt * npix * sizeof(double));
#ifdef _OPENMP
#pragma omp parallel num_threads(nt) reduction(+ : n_used, n_empty, n_window, n_qbad, sum_log)
#endif
        {
#ifdef _OPENMP
            int tid = omp_get_thread_num();
#else
            int tid = 0;
#endif
            double* rho_new = partial + (int64_t)tid * npix;
            cache_t c = {0, 0, 0};
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 256)
#endif
            for (int64_t j = 0; j < n; ++j) {
                double ey, ez, t;
                int64_t m = event_window(p, zu[j], zd[j], dl[j], &c, &n_qbad, &ey, &ez, &t);
                double D = 0.0;
                for (int64_t k = 0; k < m; ++k) {
                    int64_t i = c.idx[k];
                    double w = p->form_p ? rho[i] : s[i] * rho[i];
                    D += c.P[k] * w;
                }
                n_window += m;
                if (!(D > 0.0)) { ++n_empty; continue; }
                ++n_used;
                sum_log += log(D);
                for (int64_t k = 0; k < m; ++k) {
                    int64_t i = c.idx[k];
                    rho_new[i] += rho[i] * c.P[k] / D;
                }
            }
            free(c.idx);
            free(c.P);
        }
        double srho = 0.0;
        for (int64_t i = 0; i < npix; ++i)
            srho += p->form_p ? rho[i] : s[i] * rho[i];
        if (loglik) loglik[it] = sum_log - srho;
        for (int64_t i = 0; i < npix; ++i) {
            double v = 0.0;
            for (int k = 0; k < nt; ++k) v += partial[(int64_t)k * npix + i];
            rho[i] = v;
        }
        if (st) {
            st->n_used = n_used; st->n_empty = n_empty;
            st->n_window = n_window; st->n_qbad = n_qbad;
            double sr = 0.0;
            for (int64_t i = 0; i < npix; ++i) sr += p->form_p ? rho[i] : s[i] * rho[i];
            st->sum_s_rho = sr;
        }
    }
    free(partial);
    return 0;
}

/* Per-event denominators D_j = sum_i P_ji s_i rho_i (pass 1 only) and the
 * in-window pixel count of each event (both arrays of length n; nullable). */
int orc_denominators(const orc_params* p, const double* zu, const double* zd,
                     const double* dl, int64_t n, const double* s, const double* rho,
                     double* D_out, int64_t* count_out)
{
    int nt = nthreads_of(p);
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
        cache_t c = {0, 0, 0};
        int64_t qb = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 256)
#endif
        for (int64_t j = 0; j < n; ++j) {
            double ey, ez, t;
            int64_t m = event_window(p, zu[j], zd[j], dl[j], &c, &qb, &ey, &ez, &t);
            double D = 0.0;
            for (int64_t k = 0; k < m; ++k) D += c.P[k] * s[c.idx[k]] * rho[c.idx[k]];
            if (D_out) D_out[j] = D;
            if (count_out) count_out[j] = m;
        }
        free(c.idx);
        free(c.P);
    }
    return 0;
}

/* One MLEM update evaluated only at the listed pixels: out[k] = rho^(t+1) at
 * pixel pix[k], from Eq. iter with the current rho.  Events whose window misses
 * every listed pixel are skipped before their denominator is formed. */
/* Direct-reconstruction image (Eq. 2, Sec. 2; the paper's direct image): the
 * number of events whose reconstructed point (y~, z~) falls in each pixel.
 * Pixel (iy, iz) covers y in [-R + iy dy, -R + (iy+1) dy) and z in
 * [-L/2 + iz dz, -L/2 + (iz+1) dz); points outside the grid are not counted.
 * counts: ny*nz doubles, accumulated (the caller zeroes them). */
void orc_direct_image(const orc_params* p, const double* zu, const double* zd,
                      const double* dl, int64_t n, double* counts)
{
    for (int64_t j = 0; j < n; ++j) {
        double y, z, t;
        orc_direct(p, zu[j], zd[j], dl[j], &y, &z, &t);
        double fy = (y + p->R) / p->dy, fz = (z + 0.5 * p->L) / p->dz;
        if (!(fy >= 0.0 && fy < (double)p->ny && fz >= 0.0 && fz < (double)p->nz)) continue;
        int iy = (int)floor(fy), iz = (int)floor(fz);
        counts[(int64_t)iy * p->nz + iz] += 1.0;
    }
}

int orc_update_at_pixels(const orc_params* p, const double* zu, const double* zd,
                         const double* dl, int64_t n, const double* s, const double* rho,
                         const int64_t* pix, int32_t npx, double* out)
{
    int nt = nthreads_of(p);
    double* part = (double*)calloc((size_t)nt * npx, sizeof(double));
    /* slot[i] = the position in pix of image pixel i (its first occurrence),
     * or -1: finds a window pixel's place in the list without a search */
    int64_t npix = (int64_t)p->ny * p->nz;
    int32_t* slot = (int32_t*)malloc((size_t)npix * sizeof(int32_t));
    if (!part || !slot) {
        free(part);
        free(slot);
        return -1;
    }
    for (int64_t i = 0; i < npix; ++i) slot[i] = -1;
    for (int32_t q = npx - 1; q >= 0; --q) slot[pix[q]] = q;
    double cut2 = p->cut * p->cut;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
#ifdef _OPENMP
        int tid = omp_get_thread_num();
#else
        int tid = 0;
#endif
        cache_t c = {0, 0, 0};
        int64_t qb = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1024)
#endif
        for (int64_t j = 0; j < n; ++j) {
            double ey, ez, t;
            orc_direct(p, zu[j], zd[j], dl[j], &ey, &ez, &t);
            int hit = 0;
            for (int k = 0; k < npx && !hit; ++k) {
                int iy = (int)(pix[k] / p->nz), iz = (int)(pix[k] % p->nz);
                hit = window_bq(p, ey, ez, t, pix_y(p, iy), pix_z(p, iz)) <= cut2;
            }
            if (!hit) continue;
            int64_t m = event_window(p, zu[j], zd[j], dl[j], &c, &qb, &ey, &ez, &t);
            double D = 0.0;
            for (int64_t k = 0; k < m; ++k) D += c.P[k] * s[c.idx[k]] * rho[c.idx[k]];
            if (!(D > 0.0)) continue;
            for (int64_t k = 0; k < m; ++k) {
                int32_t q = slot[c.idx[k]];
                if (q >= 0) part[(int64_t)tid * npx + q] += rho[pix[q]] * c.P[k] / D;
            }
        }
        free(c.idx);
        free(c.P);
    }
    for (int q = 0; q < npx; ++q) {
        double v = 0.0;
        int32_t q0 = slot[pix[q]];     /* a repeated pixel takes its first entry's sum */
        for (int k = 0; k < nt; ++k) v += part[(int64_t)k * npx + q0];
        out[q] = v;
    }
    free(part);
    free(slot);
    return 0;
}

/* List-mode Poisson log-likelihood L = sum_j log D_j - sum_i s_i rho_i (events
 * with D_j = 0 are skipped, R10) and its gradient with the windows frozen at the
 * window sigmas:
 *   dL/drho_l   = s_l (sum_j P_jl / D_j - 1)
 *   dL/dsigma_k = sum_j (1/D_j) sum_i s_i rho_i P_ji d log P_ji / d sigma_k.
 * g_rho (npix) and g_sigma (2) are nullable. */
int orc_loglik_grad(const orc_params* p, const double* zu, const double* zd,
                    const double* dl, int64_t n, const double* s, const double* rho,
                    double* L_out, double* g_rho, double* g_sigma)
{
    int64_t npix = (int64_t)p->ny * p->nz;
    int nt = nthreads_of(p);
    double* part = g_rho ? (double*)calloc((size_t)nt * npix, sizeof(double)) : NULL;
    if (g_rho && !part) return -1;
    double sum_log = 0.0, gs0 = 0.0, gs1 = 0.0;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt) reduction(+ : sum_log, gs0, gs1)
#endif
    {
#ifdef _OPENMP
        int tid = omp_get_thread_num();
#else
        int tid = 0;
#endif
        cache_t c = {0, 0, 0};
        int64_t qb = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 256)
#endif
        for (int64_t j = 0; j < n; ++j) {
            double ey, ez, t;
            int64_t m = event_window(p, zu[j], zd[j], dl[j], &c, &qb, &ey, &ez, &t);
            double D = 0.0;
            for (int64_t k = 0; k < m; ++k) D += c.P[k] * s[c.idx[k]] * rho[c.idx[k]];
            if (!(D > 0.0)) continue;
            sum_log += log(D);
            if (part)
                for (int64_t k = 0; k < m; ++k)
                    part[(int64_t)tid * npix + c.idx[k]] += c.P[k] / D;
            if (g_sigma) {
                double e0 = 0.0, e1 = 0.0;
                for (int64_t k = 0; k < m; ++k) {
                    int64_t i = c.idx[k];
                    if (c.P[k] == 0.0) continue;
                    double dlg[2];
                    kernel_dlog(p, ey, ez, t, pix_y(p, (int)(i / p->nz)),
                                pix_z(p, (int)(i % p->nz)), dlg);
                    double w = s[i] * rho[i] * c.P[k];
                    e0 += w * dlg[0];
                    e1 += w * dlg[1];
                }
                gs0 += e0 / D;
                gs1 += e1 / D;
            }
        }
        free(c.idx);
        free(c.P);
    }
    double srho = 0.0;
    for (int64_t i = 0; i < npix; ++i) srho += s[i] * rho[i];
    if (L_out) *L_out = sum_log - srho;
    if (g_rho) {
        for (int64_t i = 0; i < npix; ++i) {
            double v = 0.0;
            for (int k = 0; k < nt; ++k) v += part[(int64_t)k * npix + i];
            g_rho[i] = s[i] * (v - 1.0);
        }
        free(part);
    }
    if (g_sigma) { g_sigma[0] = gs0; g_sigma[1] = gs1; }
    return 0;
}
