/*
 * spect_oracle.c -- plain FP64 CPU oracle for the rotation-based SPECT
 * projector of Li, Dewaraja & Fessler (arXiv 2301.09710), Section II-A.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA path is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the product
 * library never links, includes or calls it, and it shares no code, header
 * or table with the CUDA path.
 *
 * Every routine follows the paper's definitions literally, in double
 * precision, with loops in the paper's order.  The only parallelism is the
 * paper's own: independent views run on separate threads (Section II-A, the
 * paragraph after Algorithm 2).  Views are reduced in a fixed order so the
 * result does not depend on the thread count.
 *
 * Array conventions (0-based; the paper's are 1-based):
 *   x, mu   : nx*ny*nz, x(i,j,k) at i + nx*(j + ny*k)          (i fastest)
 *   psf     : px*pz*ny*nview_psf, p(a,b,j,l) at a + px*(b + pz*(j + ny*l))
 *   v       : nx*nz*nview, v(i,k,l) at i + nx*(k + nz*l)
 *   angles  : nview radians.
 *
 * Readings of points the paper leaves open (each one is listed with the
 * same wording in the design notes):
 *   R1 rotation centre c = (nx-1)/2 (pixel-grid centre).  The rotated
 *      image at output pixel (i,j) samples the input at
 *        xs = c + cos(t)(i-c) + sin(t)(j-c),
 *        ys = c - sin(t)(i-c) + cos(t)(j-c),
 *      so image content turns by +t.  At exact multiples of pi/2 the
 *      cosine and sine are taken as exact 0/+-1.
 *   R2 bilinear interpolation with zero padding: neighbours outside the
 *      grid contribute 0 (Section II-A: the rotation pads the image with zeros).
 *   R3 Eq. (1) attenuation: plane j = ny-1 is nearest the detector,
 *      S(j) = mu~(j)/2 + sum_{s>j} mu~(s), mubar = exp(-dy * S).
 *   R4 PSF blur is a true convolution with replicate padding in i and k
 *      and centre c_x = (px-1)/2, c_z = (pz-1)/2 (odd sizes only):
 *        c_j(i,k) = sum_{a,b} p(a,b,j,l) w(clamp(i-a+c_x), j, clamp(k-b+c_z)).
 *      The adjoint is computed as the literal transpose; it does NOT rely
 *      on the PSF being symmetric.
 *   R5 the depth index j of p(:,:,j,l) is the depth in the rotated frame.
 *   R13 the three-pass rotation (Section II-A names 3-pass 1D linear
 *      interpolation as the alternative to bilinear rotation, without the
 *      decomposition): theta = q*pi/2 + phi with q = nearest integer and
 *      phi in [-pi/4, pi/4]; first the exact quarter turn q (the R1
 *      convention at theta = q*pi/2), then three pull-backs, each a 1D
 *      linear interpolation with zero padding:
 *        along x at i + tan(phi/2)(j-c),
 *        along y at j - sin(phi)(i-c),
 *        along x at i + tan(phi/2)(j-c),
 *      whose composition samples at R(-phi)(p-c)+c, the R1 convention.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX3(i, j, k, n1, n2) ((size_t)(i) + (size_t)(n1) * ((size_t)(j) + (size_t)(n2) * (size_t)(k)))

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* cos/sin with exact values at multiples of pi/2 (reading R1). */
static void exact_cos_sin(double theta, double* c, double* s)
{
    double q = theta / (M_PI / 2.0);
    double r = nearbyint(q);
    if (fabs(q - r) < 1e-12) {
        long m = ((long)r % 4 + 4) % 4;
        static const double C[4] = {1.0, 0.0, -1.0, 0.0};
        static const double S[4] = {0.0, 1.0, 0.0, -1.0};
        *c = C[m];
        *s = S[m];
    } else {
        *c = cos(theta);
        *s = sin(theta);
    }
}

/* Sample position (xs, ys) for output pixel (i, j) of an n x n slice. */
static void sample_point(int n, double ct, double st, int i, int j, double* xs, double* ys)
{
    double c = 0.5 * (double)(n - 1);
    double di = (double)i - c, dj = (double)j - c;
    *xs = c + ct * di + st * dj;
    *ys = c - st * di + ct * dj;
}

/* ---------------------------------------------------------------------- */
/* Image rotation, Section II-A (bilinear, zero padding).                  */
/* out(i,j) = sum over the 4 neighbours q of (xs,ys) of W(i,j;q) in(q).    */
/* ---------------------------------------------------------------------- */
void oracle_rotate_slice(int n, double theta, const double* in, double* out)
{
    double ct, st;
    exact_cos_sin(theta, &ct, &st);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double xs, ys;
            sample_point(n, ct, st, i, j, &xs, &ys);
            int i0 = (int)floor(xs), j0 = (int)floor(ys);
            double fx = xs - i0, fy = ys - j0;
            double acc = 0.0;
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    int qi = i0 + di, qj = j0 + dj;
                    if (qi < 0 || qi >= n || qj < 0 || qj >= n) continue; /* zero padding */
                    double w = (di ? fx : 1.0 - fx) * (dj ? fy : 1.0 - fy);
                    acc += w * in[(size_t)qi + (size_t)n * qj];
                }
            out[(size_t)i + (size_t)n * j] = acc;
        }
}

/* Transpose of oracle_rotate_slice, written as a scatter:
 * out(q) += W(i,j;q) in(i,j) for every output pixel (i,j) and neighbour q. */
void oracle_rotate_adjoint_slice(int n, double theta, const double* in, double* out)
{
    double ct, st;
    exact_cos_sin(theta, &ct, &st);
    memset(out, 0, sizeof(double) * (size_t)n * n);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double xs, ys;
            sample_point(n, ct, st, i, j, &xs, &ys);
            int i0 = (int)floor(xs), j0 = (int)floor(ys);
            double fx = xs - i0, fy = ys - j0;
            double val = in[(size_t)i + (size_t)n * j];
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    int qi = i0 + di, qj = j0 + dj;
                    if (qi < 0 || qi >= n || qj < 0 || qj >= n) continue;
                    double w = (di ? fx : 1.0 - fx) * (dj ? fy : 1.0 - fy);
                    out[(size_t)qi + (size_t)n * qj] += w * val;
                }
        }
}

/* ---------------------------------------------------------------------- */
/* Three-pass rotation (reading R13).                                      */
/* ---------------------------------------------------------------------- */

/* theta = q*pi/2 + phi, q in 0..3, phi in [-pi/4, pi/4]. */
static void quarter_split(double theta, int* q, double* phi)
{
    double r = nearbyint(theta / (M_PI / 2.0));
    *phi = theta - r * (M_PI / 2.0);
    *q = (int)(((long)r % 4 + 4) % 4);
}

/* Source pixel of output (i, j) under the quarter turn q (R1 at theta = q*pi/2). */
static void quarter_source(int n, int q, int i, int j, int* si, int* sj)
{
    switch (q) {
        case 0: *si = i; *sj = j; break;
        case 1: *si = j; *sj = n - 1 - i; break;
        case 2: *si = n - 1 - i; *sj = n - 1 - j; break;
        default: *si = n - 1 - j; *sj = i; break;
    }
}

/* Sample of the 1D signal f(0..n-1) (stride st) at position u by linear
 * interpolation, zero outside. */
static double interp1(const double* f, int n, size_t st, double u)
{
    int u0 = (int)floor(u);
    double a = u - u0, acc = 0.0;
    if (u0 >= 0 && u0 < n) acc += (1.0 - a) * f[st * (size_t)u0];
    if (u0 + 1 >= 0 && u0 + 1 < n) acc += a * f[st * (size_t)(u0 + 1)];
    return acc;
}

/* Transpose of interp1: f(u0) += (1-a) val, f(u0+1) += a val (in range). */
static void interp1_adjoint(double* f, int n, size_t st, double u, double val)
{
    int u0 = (int)floor(u);
    double a = u - u0;
    if (u0 >= 0 && u0 < n) f[st * (size_t)u0] += (1.0 - a) * val;
    if (u0 + 1 >= 0 && u0 + 1 < n) f[st * (size_t)(u0 + 1)] += a * val;
}

/* out = rotation of the n x n slice `in` by theta in three 1D passes. */
void oracle_rotate3_slice(int n, double theta, const double* in, double* out)
{
    int q;
    double phi;
    quarter_split(theta, &q, &phi);
    double c = 0.5 * (double)(n - 1), t = tan(0.5 * phi), s = sin(phi);
    size_t nn = (size_t)n * n;
    double* h = malloc(sizeof(double) * nn);
    double* g = malloc(sizeof(double) * nn);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            int si, sj;
            quarter_source(n, q, i, j, &si, &sj);
            h[(size_t)i + (size_t)n * j] = in[(size_t)si + (size_t)n * sj];
        }
    for (int j = 0; j < n; ++j) /* pass 1: along x */
        for (int i = 0; i < n; ++i) g[(size_t)i + (size_t)n * j] = interp1(h + (size_t)n * j, n, 1, i + t * (j - c));
    for (int j = 0; j < n; ++j) /* pass 2: along y */
        for (int i = 0; i < n; ++i) h[(size_t)i + (size_t)n * j] = interp1(g + i, n, (size_t)n, j - s * (i - c));
    for (int j = 0; j < n; ++j) /* pass 3: along x */
        for (int i = 0; i < n; ++i) out[(size_t)i + (size_t)n * j] = interp1(h + (size_t)n * j, n, 1, i + t * (j - c));
    free(h);
    free(g);
}

/* Transpose of oracle_rotate3_slice: the passes' scatter transposes in
 * reverse order, then the inverse quarter turn (out is overwritten). */
void oracle_rotate3_adjoint_slice(int n, double theta, const double* in, double* out)
{
    int q;
    double phi;
    quarter_split(theta, &q, &phi);
    double c = 0.5 * (double)(n - 1), t = tan(0.5 * phi), s = sin(phi);
    size_t nn = (size_t)n * n;
    double* h = calloc(nn, sizeof(double));
    double* g = calloc(nn, sizeof(double));
    for (int j = 0; j < n; ++j) /* pass 3 transposed */
        for (int i = 0; i < n; ++i)
            interp1_adjoint(h + (size_t)n * j, n, 1, i + t * (j - c), in[(size_t)i + (size_t)n * j]);
    for (int j = 0; j < n; ++j) /* pass 2 transposed */
        for (int i = 0; i < n; ++i) interp1_adjoint(g + i, n, (size_t)n, j - s * (i - c), h[(size_t)i + (size_t)n * j]);
    memset(h, 0, sizeof(double) * nn);
    for (int j = 0; j < n; ++j) /* pass 1 transposed */
        for (int i = 0; i < n; ++i)
            interp1_adjoint(h + (size_t)n * j, n, 1, i + t * (j - c), g[(size_t)i + (size_t)n * j]);
    for (int j = 0; j < n; ++j) /* quarter turn transposed: a permutation */
        for (int i = 0; i < n; ++i) {
            int si, sj;
            quarter_source(n, q, i, j, &si, &sj);
            out[(size_t)si + (size_t)n * sj] = h[(size_t)i + (size_t)n * j];
        }
    free(h);
    free(g);
}

/* The slice rotation of a projector: 0 bilinear (R1, R2), 1 three-pass (R13). */
static void rotate_any(int mode, int n, double theta, const double* in, double* out)
{
    if (mode == 1)
        oracle_rotate3_slice(n, theta, in, out);
    else
        oracle_rotate_slice(n, theta, in, out);
}

static void rotate_any_adjoint(int mode, int n, double theta, const double* in, double* out)
{
    if (mode == 1)
        oracle_rotate3_adjoint_slice(n, theta, in, out);
    else
        oracle_rotate_adjoint_slice(n, theta, in, out);
}

/* ---------------------------------------------------------------------- */
/* Accumulated attenuation, Eq. (1) (reading R3), in the rotated frame.   */
/* mu_rot and mubar are nx*ny*nz arrays with the rotated-frame layout.     */
/* ---------------------------------------------------------------------- */
void oracle_attenuation(int nx, int ny, int nz, double dy, const double* mu_rot, double* mubar)
{
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < nx; ++i)
            for (int j = 0; j < ny; ++j) {
                double S = 0.5 * mu_rot[IDX3(i, j, k, nx, ny)];
                for (int s = j + 1; s < ny; ++s) S += mu_rot[IDX3(i, s, k, nx, ny)];
                mubar[IDX3(i, j, k, nx, ny)] = exp(-dy * S);
            }
}

/* ---------------------------------------------------------------------- */
/* Depth-dependent PSF blur of one (x,z) plane, reading R4.                */
/* w, out: nx*nz with (i,k) at i + nx*k.  p: px*pz with (a,b) at a+px*b.   */
/* ---------------------------------------------------------------------- */
void oracle_conv_plane(int nx, int nz, const double* w, const double* p, int px, int pz, double* out)
{
    int cx = (px - 1) / 2, cz = (pz - 1) / 2;
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < nx; ++i) {
            double acc = 0.0;
            for (int b = 0; b < pz; ++b) {
                int ks = clampi(k - b + cz, 0, nz - 1);
                for (int a = 0; a < px; ++a) {
                    int is = clampi(i - a + cx, 0, nx - 1);
                    acc += p[a + (size_t)px * b] * w[is + (size_t)nx * ks];
                }
            }
            out[i + (size_t)nx * k] = acc;
        }
}

/* Transpose of oracle_conv_plane as a literal scatter (out is overwritten). */
void oracle_conv_adjoint_plane(int nx, int nz, const double* v, const double* p, int px, int pz, double* out)
{
    int cx = (px - 1) / 2, cz = (pz - 1) / 2;
    memset(out, 0, sizeof(double) * (size_t)nx * nz);
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < nx; ++i) {
            double val = v[i + (size_t)nx * k];
            for (int b = 0; b < pz; ++b) {
                int ks = clampi(k - b + cz, 0, nz - 1);
                for (int a = 0; a < px; ++a) {
                    int is = clampi(i - a + cx, 0, nx - 1);
                    out[is + (size_t)nx * ks] += p[a + (size_t)px * b] * val;
                }
            }
        }
}

/* ---------------------------------------------------------------------- */
/* One view of Algorithm 1 (forward projector).                            */
/* ---------------------------------------------------------------------- */
static void forward_one_view(int nx, int ny, int nz, const double* x, const double* mu, double dy,
                             const double* psf_l, int px, int pz, double theta, int rot_mode, double* v_l,
                             double* xr, double* mr, double* mbar, double* wplane, double* cplane)
{
    size_t slice = (size_t)nx * ny;
    /* rotate x and mu slice by slice (each z-slice turns about the axial axis) */
    for (int k = 0; k < nz; ++k) {
        rotate_any(rot_mode, nx, theta, x + slice * k, xr + slice * k);
        rotate_any(rot_mode, nx, theta, mu + slice * k, mr + slice * k);
    }
    oracle_attenuation(nx, ny, nz, dy, mr, mbar);
    memset(v_l, 0, sizeof(double) * (size_t)nx * nz);
    for (int j = 0; j < ny; ++j) {
        /* attenuated rotated activity at depth j, as an (x,z) plane */
        for (int k = 0; k < nz; ++k)
            for (int i = 0; i < nx; ++i)
                wplane[i + (size_t)nx * k] = xr[IDX3(i, j, k, nx, ny)] * mbar[IDX3(i, j, k, nx, ny)];
        oracle_conv_plane(nx, nz, wplane, psf_l + (size_t)px * pz * j, px, pz, cplane);
        for (size_t m = 0; m < (size_t)nx * nz; ++m) v_l[m] += cplane[m];
    }
}

/* v = A x over all views.  psf has nview_psf views (1 = view-invariant).
 * rot_mode: 0 bilinear rotation, 1 three-pass rotation.
 * nthreads <= 0 uses the OpenMP default. */
void oracle_forward(int nx, int ny, int nz, int nview, const double* x, const double* mu, double dy,
                    const double* psf, int px, int pz, int nview_psf, const double* angles, double* v,
                    int nthreads, int rot_mode)
{
    size_t vol = (size_t)nx * ny * nz, plane = (size_t)nx * nz, psfv = (size_t)px * pz * ny;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        double* xr = malloc(sizeof(double) * vol);
        double* mr = malloc(sizeof(double) * vol);
        double* mb = malloc(sizeof(double) * vol);
        double* wp = malloc(sizeof(double) * plane);
        double* cp = malloc(sizeof(double) * plane);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int l = 0; l < nview; ++l) {
            const double* pl = psf + psfv * (nview_psf == 1 ? 0 : l);
            forward_one_view(nx, ny, nz, x, mu, dy, pl, px, pz, angles[l], rot_mode, v + plane * l, xr, mr, mb, wp,
                             cp);
        }
        free(xr); free(mr); free(mb); free(wp); free(cp);
    }
}

/* ---------------------------------------------------------------------- */
/* One view of Algorithm 2 (back projector) as the transpose of            */
/* forward_one_view, written out step by step in reverse order.            */
/* xpart (nx*ny*nz) receives this view's contribution (overwritten).        */
/* ---------------------------------------------------------------------- */
static void back_one_view(int nx, int ny, int nz, const double* v_l, const double* mu, double dy,
                          const double* psf_l, int px, int pz, double theta, int rot_mode, double* xpart,
                          double* mr, double* mbar, double* t, double* wbar)
{
    size_t slice = (size_t)nx * ny;
    for (int k = 0; k < nz; ++k) rotate_any(rot_mode, nx, theta, mu + slice * k, mr + slice * k);
    oracle_attenuation(nx, ny, nz, dy, mr, mbar);
    for (int j = 0; j < ny; ++j) {
        /* adjoint of (depth sum + blur at depth j): the same v plane for every j */
        oracle_conv_adjoint_plane(nx, nz, v_l, psf_l + (size_t)px * pz * j, px, pz, wbar);
        /* adjoint of the attenuation multiply (a diagonal scaling) */
        for (int k = 0; k < nz; ++k)
            for (int i = 0; i < nx; ++i)
                t[IDX3(i, j, k, nx, ny)] = wbar[i + (size_t)nx * k] * mbar[IDX3(i, j, k, nx, ny)];
    }
    /* adjoint of the rotation, slice by slice */
    for (int k = 0; k < nz; ++k) rotate_any_adjoint(rot_mode, nx, theta, t + slice * k, xpart + slice * k);
}

/* x = A' v over all views (x is overwritten).  Views run in blocks of
 * nthreads; each block's per-view parts are added in view order, so the
 * result is the same for any thread count. */
void oracle_back(int nx, int ny, int nz, int nview, const double* v, const double* mu, double dy,
                 const double* psf, int px, int pz, int nview_psf, const double* angles, double* x,
                 int nthreads, int rot_mode)
{
    size_t vol = (size_t)nx * ny * nz, plane = (size_t)nx * nz, psfv = (size_t)px * pz * ny;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    if (nthreads > nview) nthreads = nview;
    if (nthreads < 1) nthreads = 1;
    double* parts = malloc(sizeof(double) * vol * (size_t)nthreads);
    memset(x, 0, sizeof(double) * vol);
    for (int l0 = 0; l0 < nview; l0 += nthreads) {
        int nb = nview - l0 < nthreads ? nview - l0 : nthreads;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
        {
            double* mr = malloc(sizeof(double) * vol);
            double* mb = malloc(sizeof(double) * vol);
            double* t = malloc(sizeof(double) * vol);
            double* wb = malloc(sizeof(double) * plane);
#ifdef _OPENMP
#pragma omp for schedule(static, 1)
#endif
            for (int b = 0; b < nb; ++b) {
                int l = l0 + b;
                const double* pl = psf + psfv * (nview_psf == 1 ? 0 : l);
                back_one_view(nx, ny, nz, v + plane * l, mu, dy, pl, px, pz, angles[l], rot_mode, parts + vol * b, mr,
                              mb, t, wb);
            }
            free(mr); free(mb); free(t); free(wb);
        }
        for (int b = 0; b < nb; ++b)
            for (size_t m = 0; m < vol; ++m) x[m] += parts[vol * b + m];
    }
    free(parts);
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
