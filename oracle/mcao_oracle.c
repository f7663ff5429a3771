/*
 * FP64 CPU oracle of the MCAO wavefront-sensing-and-control step.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the package's smoke check and the CPU-baseline leg of
 * the benchmark load this file's shared object; the product library never links, loads or
 * calls it, and nothing here is shared with the CUDA path (no header, table or helper).
 *
 * What it computes (arXiv:1608.00386, "The closed loop" and neighbouring subsections; the
 * paper prints no equations, so each step is the plain definition of the quantity it names):
 *   a1  frozen-flow offset of every layer, o_l = (k dt) v_l            ("The atmospheric layers
 *       generation": static screens, frozen flow)
 *   a2  DM surface S_m(x) = sum_j c_j exp(-|x-x_j|^2 / 2 sigma^2), g(pitch) = coupling
 *                                                                       ("Influence function and
 *       modal base": DM = linear combination of analytic influence functions)
 *   a3  residual phase along each guide star: bilinear samples of every layer at the cone-beam
 *       projected point minus the same samples of every DM surface   ("The open loop wave-front
 *       measurements": geometric projection, LGS at finite distance; "The closed loop":
 *       residual = open-loop WF minus DM)
 *   a4-a7 Shack-Hartmann spot: field A exp(i phi) zero-padded to N_fft, 2-D FFT, |.|^2,
 *       sodium elongation as FFT * analytic Gaussian OTF * inverse FFT, fftshift, b x b bin,
 *       flux normalisation                                            ("The closed loop": WFS
 *       modules compute X and Y slopes from the residual phase)
 *   a8  photon + read noise from a counter-based Philox4x32-10 stream
 *   a9  centre-of-gravity slopes minus the reference slopes ("The calibration of the interaction
 *       matrices": reference slope vector)
 *   a10-a11 Delta c = R s (plain double loop), c <- c + g Delta c ("The closed loop": slopes times
 *       control matrix give differential coefficients added to the mirror; pure integrator).
 *       Reduced-precision variants replace each R_ij by its bfloat16 or FP8-E4M3 (per-row scale)
 *       value, defined by the quantizers below; the product itself stays in double.
 *   a12 science residual along each science direction: instantaneous on-axis Strehl
 *       |sum A e^{i phi}|^2 / (sum A)^2 and the long-exposure PSF |FFT(pad(A e^{i phi}))|^2
 *       accumulated in double                                           ("The Point Spread
 *       Functions (PSFs)")
 * Beyond the per-step path, with the same conventions:
 *   - second-order controller, Marechal Strehl exp(-sigma^2), sodium-layer updates ("The
 *     closed loop", "The Point Spread Functions (PSFs)");
 *   - von Karman phase-screen coefficients and amplitudes of the FFT method ("The atmospheric
 *     layers generation"; the inverse DFT is numpy's, in oracle/__init__.py);
 *   - DM misregistration: the surface of a translated, rotated and magnified DM by the direct
 *     sum over actuators ("Conclusions": rotation of the DM and its modal basis);
 *   - the interaction matrix as a derivative is central differences of this file's noise-free
 *     measurement (oracle/__init__.py: jacobian_fd, subap_jacobian_fd).
 *
 * Readings of the points the paper leaves open (coordinates, units, centring ramp, elongation
 * geometry, noise sampler) follow one fixed list; each function below states the reading it
 * applies.  Precision: everything in double except the noise sampler, which by definition runs
 * in float with an explicit operation order so that a float intensity maps to one integer.
 *
 * Parity status per function: every stage is pinned by closed-form tests (Dirichlet spot,
 * Parseval, exact roll under an integer tilt, affine exactness of bilinear sampling, Gaussian
 * poke, periodised-Gaussian elongation kernel, numpy cross-checks of FFT, matmul and the DM
 * sum, Strehl of a flat wavefront, Marechal regime, integrator recursion, controller error
 * recursion, von Karman structure function and its Kolmogorov limit, screen and noise moments,
 * piston invariance and step halving of the derivatives, rigid-body identities of the moved
 * DM).  The one exception is Philox4x32-10, pinned against an independent implementation
 * (cuRAND's) only on a GPU.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------------------------ */
/* configuration structs (mirrored by ctypes in oracle/__init__.py)                            */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int type;                 /* 0 = natural guide star (at infinity), 1 = laser guide star     */
    int n_sub, n_px, n_fft, n_bin;
    int pad_;
    double theta_x, theta_y;  /* direction, rad                                                  */
    double height;            /* LGS height above the telescope, m (ignored for NGS)            */
    double lambda;            /* sensing wavelength, m                                           */
    double n_photons;         /* photons per fully illuminated subaperture per frame            */
    double read_noise;        /* e- rms per detector pixel                                       */
    double valid_thr;         /* minimum illuminated fraction of a valid subaperture            */
    double na_fwhm;           /* sodium layer FWHM thickness, m (0 = no elongation)              */
    double launch_x, launch_y;/* laser launch position in the pupil, m                          */
} orc_wfs;

typedef struct {
    int n_px, pad;            /* pupil samples across D; zero-pad factor of the PSF FFT         */
    double theta_x, theta_y, lambda;
} orc_sci;

typedef struct {
    int n;                    /* screen is n x n, periodic                                       */
    int pad_;
    double pixel, alt, vx, vy;/* m, m, m/s, m/s                                                  */
    const float* phase;       /* rad at the reference wavelength, row-major [y][x]              */
} orc_layer;

typedef struct {
    int nx, ny, surf_n, pad_;
    double alt, pitch, coupling, surf_dx;
    const uint8_t* valid;     /* [ny][nx] actuator validity                                      */
} orc_dm;

typedef struct {
    double D, obstruction, lambda_ref, dt, gain;
    uint64_t seed;
    int noise, psf_every;
    int n_wfs, n_sci, n_layers, n_dms;
    const orc_wfs* wfs;
    const orc_sci* sci;
    const orc_layer* layers;
    const orc_dm* dms;
    int n_cmd, n_slopes;
    const float* R;           /* [n_cmd][n_slopes] row-major, kept by reference                 */
    const float* s_ref;       /* [n_slopes]                                                       */
    int r_dtype;              /* 0: R as given; 1: R rounded to bfloat16; 2: FP8 E4M3 with a
                                 float scale per row (the reduced-precision product variants)    */
} orc_config;

/* ------------------------------------------------------------------------------------------ */
/* FFT: mixed-radix Cooley-Tukey by direct recursion on the smallest prime factor              */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int n;
    double* wr; double* wi;   /* w[j] = exp(-2 pi i j / n)                                       */
} orc_plan;

static orc_plan* plan_new(int n) {
    orc_plan* p = (orc_plan*)calloc(1, sizeof(orc_plan));
    p->n = n;
    p->wr = (double*)malloc(sizeof(double) * n);
    p->wi = (double*)malloc(sizeof(double) * n);
    for (int j = 0; j < n; ++j) {
        double a = -2.0 * ORC_PI * (double)j / (double)n;
        p->wr[j] = cos(a);
        p->wi[j] = sin(a);
    }
    return p;
}
static void plan_free(orc_plan* p) { if (p) { free(p->wr); free(p->wi); free(p); } }

static int smallest_factor(int n) {
    for (int p = 2; p * p <= n; ++p) if (n % p == 0) return p;
    return n;
}

/* y[k] = sum_j x[j*xs] W_n^{jk}, W_n = exp(-+2 pi i / n); twiddles read from the plan of size
 * P->n with stride tstep = P->n / n.  tmp holds n values while combining. */
static void fft_rec(int n, const double* xr, const double* xi, int xs, double* yr, double* yi,
                    const orc_plan* P, int tstep, int inverse, double* tr, double* ti) {
    if (n == 1) { yr[0] = xr[0]; yi[0] = xi[0]; return; }
    int p = smallest_factor(n), m = n / p;
    for (int r = 0; r < p; ++r)
        fft_rec(m, xr + r * xs, xi + r * xs, xs * p, yr + r * m, yi + r * m, P, tstep * p, inverse, tr, ti);
    for (int k = 0; k < n; ++k) {
        int q = k % m;
        double ar = 0.0, ai = 0.0;
        for (int r = 0; r < p; ++r) {
            int idx = (int)(((long)r * k) % n) * tstep;
            double wr = P->wr[idx], wi = inverse ? -P->wi[idx] : P->wi[idx];
            double vr = yr[r * m + q], vi = yi[r * m + q];
            ar += vr * wr - vi * wi;
            ai += vr * wi + vi * wr;
        }
        tr[k] = ar; ti[k] = ai;
    }
    memcpy(yr, tr, sizeof(double) * n);
    memcpy(yi, ti, sizeof(double) * n);
}

/* in-place 1-D DFT of length P->n; inverse includes the 1/n factor */
static void fft1_plan(const orc_plan* P, double* re, double* im, int inverse, double* ws) {
    int n = P->n;
    double *xr = ws, *xi = ws + n, *tr = ws + 2 * n, *ti = ws + 3 * n;
    memcpy(xr, re, sizeof(double) * n);
    memcpy(xi, im, sizeof(double) * n);
    fft_rec(n, xr, xi, 1, re, im, P, 1, inverse, tr, ti);
    if (inverse) for (int k = 0; k < n; ++k) { re[k] /= n; im[k] /= n; }
}

/* in-place 2-D DFT of an n x n row-major array: every row, then every column */
static void fft2_plan(const orc_plan* P, double* re, double* im, int inverse, double* ws) {
    int n = P->n;
    double *cr = ws + 4 * n, *ci = ws + 5 * n;
    for (int y = 0; y < n; ++y) fft1_plan(P, re + (size_t)y * n, im + (size_t)y * n, inverse, ws);
    for (int x = 0; x < n; ++x) {
        for (int y = 0; y < n; ++y) { cr[y] = re[(size_t)y * n + x]; ci[y] = im[(size_t)y * n + x]; }
        fft1_plan(P, cr, ci, inverse, ws);
        for (int y = 0; y < n; ++y) { re[(size_t)y * n + x] = cr[y]; im[(size_t)y * n + x] = ci[y]; }
    }
}

void orc_fft1(int n, double* re, double* im, int inverse) {
    orc_plan* P = plan_new(n);
    double* ws = (double*)malloc(sizeof(double) * 6 * n);
    fft1_plan(P, re, im, inverse, ws);
    free(ws); plan_free(P);
}

void orc_fft2(int n, double* re, double* im, int inverse) {
    orc_plan* P = plan_new(n);
    double* ws = (double*)malloc(sizeof(double) * 6 * n);
    fft2_plan(P, re, im, inverse, ws);
    free(ws); plan_free(P);
}

/* ------------------------------------------------------------------------------------------ */
/* geometry                                                                                   */
/* ------------------------------------------------------------------------------------------ */

/* Pupil amplitude on an n x n grid across D: sample i sits at (i - (n-1)/2) D/n; amplitude 1
 * inside the annulus obstruction*D/2 <= r <= D/2, else 0 (binary pupil sampled at centres). */
void orc_pupil(double D, double obstruction, int n, double* A) {
    double d = D / (double)n, R2 = 0.25 * D * D, r2o = 0.25 * obstruction * obstruction * D * D;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double x = ((double)i - 0.5 * (double)(n - 1)) * d;
            double y = ((double)j - 0.5 * (double)(n - 1)) * d;
            double r2 = x * x + y * y;
            A[(size_t)j * n + i] = (r2 <= R2 && r2 >= r2o) ? 1.0 : 0.0;
        }
}

/* Valid subapertures ("selecting the valid sub-aperture", Control Matrix subsection): the
 * illuminated fraction sum(A)/n_px^2 of a subaperture must reach thr.  valid[n_sub^2] gets 0/1,
 * frac[n_sub^2] the fraction; returns the number of valid subapertures. */
int orc_valid_subaps(const double* A, int n_sub, int n_px, double thr, int* valid, double* frac) {
    int n = n_sub * n_px, count = 0;
    for (int sy = 0; sy < n_sub; ++sy)
        for (int sx = 0; sx < n_sub; ++sx) {
            double s = 0.0;
            for (int y = 0; y < n_px; ++y)
                for (int x = 0; x < n_px; ++x) s += A[(size_t)(sy * n_px + y) * n + sx * n_px + x];
            double f = s / (double)(n_px * n_px);
            frac[sy * n_sub + sx] = f;
            valid[sy * n_sub + sx] = (f >= thr) ? 1 : 0;
            count += valid[sy * n_sub + sx];
        }
    return count;
}

static long wrap_index(long i, long n) { long r = i % n; return r < 0 ? r + n : r; }

/* Bilinear sample of a periodic n x n screen at fractional grid index (fx, fy). */
double orc_bilinear_periodic(const double* s, int n, double fx, double fy) {
    double flx = floor(fx), fly = floor(fy);
    double tx = fx - flx, ty = fy - fly;
    long ix = (long)flx, iy = (long)fly;
    long x0 = wrap_index(ix, n), x1 = wrap_index(ix + 1, n);
    long y0 = wrap_index(iy, n), y1 = wrap_index(iy + 1, n);
    return (1.0 - tx) * (1.0 - ty) * s[y0 * n + x0] + tx * (1.0 - ty) * s[y0 * n + x1]
         + (1.0 - tx) * ty * s[y1 * n + x0] + tx * ty * s[y1 * n + x1];
}

/* Bilinear sample of a bounded n x n grid; the index is clamped into [0, n-1] first, so points
 * beyond the grid take the edge value. */
double orc_bilinear_clamped(const double* s, int n, double fx, double fy) {
    if (fx < 0.0) fx = 0.0;
    if (fy < 0.0) fy = 0.0;
    if (fx > (double)(n - 1)) fx = (double)(n - 1);
    if (fy > (double)(n - 1)) fy = (double)(n - 1);
    long ix = (long)floor(fx), iy = (long)floor(fy);
    if (ix > n - 2) ix = n - 2;
    if (iy > n - 2) iy = n - 2;
    double tx = fx - (double)ix, ty = fy - (double)iy;
    return (1.0 - tx) * (1.0 - ty) * s[iy * n + ix] + tx * (1.0 - ty) * s[iy * n + ix + 1]
         + (1.0 - tx) * ty * s[(iy + 1) * n + ix] + tx * ty * s[(iy + 1) * n + ix + 1];
}

/* ------------------------------------------------------------------------------------------ */
/* DM surface (a2)                                                                            */
/* ------------------------------------------------------------------------------------------ */

/* Gaussian influence function width: exp(-pitch^2 / 2 sigma^2) = coupling. */
double orc_if_sigma(double pitch, double coupling) { return pitch / sqrt(2.0 * log(1.0 / coupling)); }

/* S[j][i] = sum_{a,b} C[b][a] g(x_i - x_a) g(y_j - y_b) over the actuator grid (C zero at
 * invalid actuators), evaluated as the product Gy C Gx^T, which equals the direct double sum
 * because the Gaussian factorises (no truncation). */
void orc_dm_surface(int nx, int ny, double pitch, double coupling, int surf_n, double surf_dx,
                    const double* C, double* S) {
    double sig = orc_if_sigma(pitch, coupling);
    double* Gx = (double*)malloc(sizeof(double) * (size_t)surf_n * nx);
    double* Gy = (double*)malloc(sizeof(double) * (size_t)surf_n * ny);
    double* T = (double*)malloc(sizeof(double) * (size_t)ny * surf_n);
    for (int i = 0; i < surf_n; ++i) {
        double x = ((double)i - 0.5 * (double)(surf_n - 1)) * surf_dx;
        for (int a = 0; a < nx; ++a) {
            double xa = ((double)a - 0.5 * (double)(nx - 1)) * pitch;
            Gx[(size_t)i * nx + a] = exp(-(x - xa) * (x - xa) / (2.0 * sig * sig));
        }
        for (int b = 0; b < ny; ++b) {
            double yb = ((double)b - 0.5 * (double)(ny - 1)) * pitch;
            Gy[(size_t)i * ny + b] = exp(-(x - yb) * (x - yb) / (2.0 * sig * sig));
        }
    }
    /* T[b][i] = sum_a C[b][a] Gx[i][a] */
    for (int b = 0; b < ny; ++b)
        for (int i = 0; i < surf_n; ++i) {
            double acc = 0.0;
            for (int a = 0; a < nx; ++a) acc += C[(size_t)b * nx + a] * Gx[(size_t)i * nx + a];
            T[(size_t)b * surf_n + i] = acc;
        }
    /* S[j][i] = sum_b Gy[j][b] T[b][i] */
    for (int j = 0; j < surf_n; ++j)
        for (int i = 0; i < surf_n; ++i) {
            double acc = 0.0;
            for (int b = 0; b < ny; ++b) acc += Gy[(size_t)j * ny + b] * T[(size_t)b * surf_n + i];
            S[(size_t)j * surf_n + i] = acc;
        }
    free(Gx); free(Gy); free(T);
}

/* Surface of a misregistered DM: the DM's own surface function evaluated at T^-1(x, y), where
 * T(q) = mag R(rot) q + (shift_x, shift_y) maps DM coordinates to the beam's (rotation
 * counter-clockwise by rot): S(x, y) = sum_{a,b} C[b][a] exp(-|T^-1(x, y) - (x_a, y_b)|^2 / 2 sigma^2),
 * the direct double sum over every actuator (the DM translated, rotated and magnified as a rigid
 * body with its influence functions). */
void orc_dm_surface_misreg(int nx, int ny, double pitch, double coupling, int surf_n, double surf_dx,
                           double shift_x, double shift_y, double rot, double mag, const double* C, double* S) {
    double sig = orc_if_sigma(pitch, coupling);
    double cr = cos(rot), sr = sin(rot);
    for (int j = 0; j < surf_n; ++j)
        for (int i = 0; i < surf_n; ++i) {
            double x = ((double)i - 0.5 * (double)(surf_n - 1)) * surf_dx - shift_x;
            double y = ((double)j - 0.5 * (double)(surf_n - 1)) * surf_dx - shift_y;
            double qx = (cr * x + sr * y) / mag, qy = (-sr * x + cr * y) / mag;
            double acc = 0.0;
            for (int b = 0; b < ny; ++b) {
                double yb = ((double)b - 0.5 * (double)(ny - 1)) * pitch;
                for (int a = 0; a < nx; ++a) {
                    double xa = ((double)a - 0.5 * (double)(nx - 1)) * pitch;
                    double d2 = (qx - xa) * (qx - xa) + (qy - yb) * (qy - yb);
                    acc += C[(size_t)b * nx + a] * exp(-d2 / (2.0 * sig * sig));
                }
            }
            S[(size_t)j * surf_n + i] = acc;
        }
}

/* ------------------------------------------------------------------------------------------ */
/* Shack-Hartmann spot (a4-a7) and centroid (a9)                                              */
/* ------------------------------------------------------------------------------------------ */

/* Sodium elongation OTF at signed frequency (ux, uy) of an N-point grid: the Fourier transform
 * of a Gaussian of standard deviation sigma_pix image pixels along the unit direction (dx, dy),
 * exp(-2 pi^2 sigma^2 (f . d)^2) with f = u / N cycles per pixel. */
static double na_otf(int ux, int uy, int N, double sigma_pix, double dx, double dy) {
    double f = ((double)ux * dx + (double)uy * dy) / (double)N;
    return exp(-2.0 * ORC_PI * ORC_PI * sigma_pix * sigma_pix * f * f);
}

/* Shifted (centred) high-resolution spot image of one subaperture, n_fft x n_fft, before
 * binning and before flux normalisation.
 *   E[y][x] = A exp(i (phi - pi (x + y) / N)) for x, y < n_px, 0 elsewhere (half-bin centring
 *   ramp: a flat wavefront puts the spot centre at index N/2 - 1/2 after the shift);
 *   I = |FFT2(E)|^2;  if sigma_pix > 0: I <- Re IFFT2(FFT2(I) * OTF);  I_s[j] = I[(j + N/2) mod N].
 * phase is in rad at the sensing wavelength, [n_px][n_px] row-major. */
static void sh_image_plan(int n_px, const orc_plan* P, const double* amp, const double* phase,
                          double sigma_pix, double dx, double dy, double* img, double* work) {
    int N = P->n;
    double *er = work, *ei = work + (size_t)N * N, *ws = work + (size_t)2 * N * N;
    memset(er, 0, sizeof(double) * (size_t)N * N);
    memset(ei, 0, sizeof(double) * (size_t)N * N);
    for (int y = 0; y < n_px; ++y)
        for (int x = 0; x < n_px; ++x) {
            double a = amp[y * n_px + x];
            double ph = phase[y * n_px + x] - ORC_PI * (double)(x + y) / (double)N;
            er[(size_t)y * N + x] = a * cos(ph);
            ei[(size_t)y * N + x] = a * sin(ph);
        }
    fft2_plan(P, er, ei, 0, ws);
    for (size_t q = 0; q < (size_t)N * N; ++q) {
        er[q] = er[q] * er[q] + ei[q] * ei[q];
        ei[q] = 0.0;
    }
    if (sigma_pix > 0.0) {
        fft2_plan(P, er, ei, 0, ws);
        for (int ky = 0; ky < N; ++ky)
            for (int kx = 0; kx < N; ++kx) {
                int ux = kx < N / 2 ? kx : kx - N, uy = ky < N / 2 ? ky : ky - N;
                double o = na_otf(ux, uy, N, sigma_pix, dx, dy);
                er[(size_t)ky * N + kx] *= o;
                ei[(size_t)ky * N + kx] *= o;
            }
        fft2_plan(P, er, ei, 1, ws);
    }
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i)
            img[(size_t)j * N + i] = er[(size_t)((j + N / 2) % N) * N + (i + N / 2) % N];
}

void orc_sh_image(int n_px, int n_fft, const double* amp, const double* phase, double sigma_pix,
                  double dx, double dy, double* img) {
    orc_plan* P = plan_new(n_fft);
    double* work = (double*)malloc(sizeof(double) * ((size_t)2 * n_fft * n_fft + 6 * n_fft));
    sh_image_plan(n_px, P, amp, phase, sigma_pix, dx, dy, img, work);
    free(work); plan_free(P);
}

/* b x b binning of the centred image: out[m][n] = sum of img over rows b m .. b m + b - 1 and
 * columns b n .. b n + b - 1. */
void orc_bin(int n_fft, int n_bin, const double* img, double* out) {
    int nd = n_fft / n_bin;
    for (int my = 0; my < nd; ++my)
        for (int mx = 0; mx < nd; ++mx) {
            double s = 0.0;
            for (int ty = 0; ty < n_bin; ++ty)
                for (int tx = 0; tx < n_bin; ++tx)
                    s += img[(size_t)(my * n_bin + ty) * n_fft + mx * n_bin + tx];
            out[my * nd + mx] = s;
        }
}

/* Centre of gravity in detector pixels, x_i = i - (n_det - 1)/2; no threshold, no window; a
 * frame whose total is not positive gives zero slopes. */
void orc_cog(int n_det, const double* img, double* sx, double* sy) {
    double s = 0.0, mx = 0.0, my = 0.0, c = 0.5 * (double)(n_det - 1);
    for (int y = 0; y < n_det; ++y)
        for (int x = 0; x < n_det; ++x) {
            double v = img[y * n_det + x];
            s += v; mx += ((double)x - c) * v; my += ((double)y - c) * v;
        }
    if (s > 0.0) { *sx = mx / s; *sy = my / s; } else { *sx = 0.0; *sy = 0.0; }
}

/* ------------------------------------------------------------------------------------------ */
/* Noise (a8): Philox4x32-10 and a float sampler with a fixed operation order                 */
/* ------------------------------------------------------------------------------------------ */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11): ten rounds of two 32x32->64 multiplications with the round keys bumped by the Weyl
 * constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (r < 9) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform in (0, 1): (w >> 8) + 1/2, times 2^-24 (exact in float) */
float orc_uniform_f32(uint32_t w) { return ((float)(w >> 8) + 0.5f) * 5.9604644775390625e-8f; }

static float f32_from_bits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t bits_from_f32(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* exp(x) in float for x in [-87, 0]: Cody-Waite reduction x = k ln2 + r (ln2 split into a
 * short high part and a correction), Taylor polynomial of degree 7 for exp(r) on |r| <= ln2/2
 * by Horner with fused multiply-adds, then scaling by 2^k through the exponent field. */
float orc_exp_f32(float x) {
    const float log2e = 1.44269502f, ln2_hi = 0.693145752f, ln2_lo = 1.42860677e-06f;
    float kf = rintf(x * log2e);
    float r = fmaf(-kf, ln2_hi, x);
    r = fmaf(-kf, ln2_lo, r);
    float p = 1.0f / 5040.0f;
    p = fmaf(p, r, 1.0f / 720.0f);
    p = fmaf(p, r, 1.0f / 120.0f);
    p = fmaf(p, r, 1.0f / 24.0f);
    p = fmaf(p, r, 1.0f / 6.0f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int k = (int)kf;
    if (k < -126) return 0.0f;
    return p * f32_from_bits((uint32_t)(k + 127) << 23);
}

/* log(u) in float for normal u > 0: u = m 2^e with m in [sqrt(1/2), sqrt(2)), then
 * log m = 2 atanh(s), s = (m - 1) fl(1/(m + 1)) (a correctly rounded reciprocal, then a
 * product), by its odd series to s^9. */
float orc_log_f32(float u) {
    uint32_t b = bits_from_f32(u);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = f32_from_bits((b & 0x007fffffu) | 0x3f800000u);
    if (m > 1.41421356f) { m = m * 0.5f; e += 1; }
    float rcp = 1.0f / (m + 1.0f);
    float s = (m - 1.0f) * rcp;
    float s2 = s * s;
    float p = 1.0f / 9.0f;
    p = fmaf(p, s2, 1.0f / 7.0f);
    p = fmaf(p, s2, 1.0f / 5.0f);
    p = fmaf(p, s2, 1.0f / 3.0f);
    p = fmaf(p, s2, 1.0f);
    float lm = 2.0f * s * p;
    const float ln2_hi = 0.693145752f, ln2_lo = 1.42860677e-06f;
    float ef = (float)e;
    return fmaf(ef, ln2_hi, fmaf(ef, ln2_lo, lm));
}

/* Taylor polynomials of sin and cos on |y| <= pi/4 */
static float sin_poly(float y) {
    float y2 = y * y;
    float p = 1.0f / 362880.0f;
    p = fmaf(p, y2, -1.0f / 5040.0f);
    p = fmaf(p, y2, 1.0f / 120.0f);
    p = fmaf(p, y2, -1.0f / 6.0f);
    return fmaf(p * y2, y, y);
}
static float cos_poly(float y) {
    float y2 = y * y;
    float p = 1.0f / 40320.0f;
    p = fmaf(p, y2, -1.0f / 720.0f);
    p = fmaf(p, y2, 1.0f / 24.0f);
    p = fmaf(p, y2, -0.5f);
    return fmaf(p, y2, 1.0f);
}

/* cos(2 pi u) and sin(2 pi u) for u in [0, 1]: quadrant q = rint(4u), y = 2 pi (u - q/4) in
 * [-pi/4, pi/4] (u - q/4 is exact: for q > 0, q/4 and u are within a factor 2 of each other),
 * then cos(y + q pi/2) and sin(y + q pi/2) from the two polynomials by quadrant. */
void orc_sincos2pi_f32(float u, float* c, float* s) {
    const float twopi = 6.28318548f;
    float qf = rintf(4.0f * u);
    float y = (u - 0.25f * qf) * twopi;
    float sp = sin_poly(y), cp = cos_poly(y);
    switch (((int)qf) & 3) {
        case 0: *c = cp; *s = sp; break;
        case 1: *c = -sp; *s = cp; break;
        case 2: *c = -cp; *s = -sp; break;
        default: *c = sp; *s = -cp; break;
    }
}

/* Two independent standard normals by Box-Muller from two uniforms:
 * r = sqrt(-2 log u0), (r cos 2 pi u1, r sin 2 pi u1). */
static void box_muller2(float u0, float u1, float* zc, float* zs) {
    float rad = sqrtf(-2.0f * orc_log_f32(u0));
    float c, s;
    orc_sincos2pi_f32(u1, &c, &s);
    *zc = rad * c;
    *zs = rad * s;
}

/* Phase-screen amplitudes ("The atmospheric layers generation": screens drawn from the
 * turbulence spectrum), the FFT method on an n x n periodic grid of pitch `pixel` (m):
 * frequency (fx, fy) = (kx', ky') / (n pixel) cycles/m with kx' = kx for kx <= (n-1)/2 and
 * kx - n above; von Karman phase spectrum PSD = 0.023 r0^(-5/3) (f^2 + L0^-2)^(-11/6);
 * a_k = sqrt(PSD) / (n pixel) (the square root of PSD times the frequency cell), a_0 = 0.
 * Output amp: [n][n] row-major by (ky, kx). */
void orc_screen_amp(int n, double pixel, double r0, double L0, double* amp) {
    const double df = 1.0 / (n * pixel);
    for (int ky = 0; ky < n; ++ky) {
        for (int kx = 0; kx < n; ++kx) {
            const int sx = (kx <= (n - 1) / 2) ? kx : kx - n;
            const int sy = (ky <= (n - 1) / 2) ? ky : ky - n;
            const double fx = sx * df, fy = sy * df;
            double a = 0.0;
            if (kx != 0 || ky != 0) {
                const double psd = 0.023 * pow(r0, -5.0 / 3.0) * pow(fx * fx + fy * fy + 1.0 / (L0 * L0), -11.0 / 6.0);
                a = sqrt(psd) * df;
            }
            amp[(size_t)ky * n + kx] = a;
        }
    }
}

/* Phase-screen coefficients c_k = (z_c + i z_s) a_k, with (z_c, z_s) the Box-Muller pair of
 * Philox4x32-10 words 0 and 1 for counter (k low 32 bits, k high 32 bits, 0, 1), key = seed,
 * k = ky n + kx.  The screen is Re sum_k c_k exp(2 pi i (kx x + ky y) / n), formed by the
 * caller.  Output re/im: [n][n] row-major by (ky, kx). */
void orc_screen_coeffs(int n, double pixel, double r0, double L0, uint64_t seed, double* re, double* im) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_screen_amp(n, pixel, r0, L0, re);
    for (uint64_t k = 0; k < (uint64_t)n * (uint64_t)n; ++k) {
        const uint32_t ctr[4] = {(uint32_t)k, (uint32_t)(k >> 32), 0u, 1u};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        float zc, zs;
        box_muller2(orc_uniform_f32(w[0]), orc_uniform_f32(w[1]), &zc, &zs);
        const double a = re[k];
        re[k] = (double)zc * a;
        im[k] = (double)zs * a;
    }
}

/* One noisy detector pixel: photon count ~ Poisson(lambda) plus rint(read_noise * z_c).
 * Words 2 and 3 give one Box-Muller pair (z_c, z_s), computed when read_noise > 0 or
 * lambda >= 16.  lambda < 16: inversion with p_0 = exp(-lambda), p_{k+1} = p_k q_{k+1},
 * q_j = fl(lambda fl(1/j)) (the ratio formed first, then the product), smallest k with
 * u <= F_k, k capped at 64, u from word 0.  lambda >= 16: max(0, rint(lambda + sqrt(lambda) z_s)).
 * Counter = (c0, c1, c2, 0), key = (seed low word, seed high word). */
/* Photon count of one pixel: Poisson by inversion for lambda < 16 (the smallest k with
 * u <= F_k, p_0 = exp(-lambda), p_k = p_{k-1} fl(lambda fl(1/k)), k <= 64), else
 * max(0, rint(lambda + sqrt(lambda) y)) with the standard normal y. */
static int photons_f32(float lam, float u, float y) {
    if (lam < 16.0f) {
        float p = orc_exp_f32(-lam), F = p;
        int k = 0;
        while (F < u && k < 64) {
            k += 1;
            float q = lam * (1.0f / (float)k);
            p = p * q;
            F = F + p;
        }
        return k;
    }
    int n = (int)lrintf(fmaf(sqrtf(lam), y, lam));
    return n < 0 ? 0 : n;
}

/* Noisy counts of a pixel pair (pixels o and o + n_det^2/2 of one subaperture frame; c0 the frame
 * index of pixel o, c1 the step, c2 the sensor): draw A = Philox(c0, c1, c2, 0) gives the two
 * inversion uniforms (words 0 and 1) and, with read noise, one Box-Muller pair (words 2, 3) whose
 * outputs are the two pixels' read noise rint(sigma z); draw B = Philox(c0, c1, c2, 2), used only
 * when a pixel has lambda >= 16, gives one Box-Muller pair (words 2, 3) for the photon normals. */
void orc_noise_pair(float lam_a, float lam_b, float read_noise, uint32_t c0, uint32_t c1, uint32_t c2, uint64_t seed,
                    int32_t* na, int32_t* nb) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ca[4] = {c0, c1, c2, 0u}, wa[4];
    orc_philox4x32_10(ca, key, wa);
    float ya = 0.0f, yb = 0.0f;
    if (!(lam_a < 16.0f) || !(lam_b < 16.0f)) {
        uint32_t cb[4] = {c0, c1, c2, 2u}, wb[4];
        orc_philox4x32_10(cb, key, wb);
        box_muller2(orc_uniform_f32(wb[2]), orc_uniform_f32(wb[3]), &ya, &yb);
    }
    int a = photons_f32(lam_a, orc_uniform_f32(wa[0]), ya);
    int b = photons_f32(lam_b, orc_uniform_f32(wa[1]), yb);
    if (read_noise > 0.0f) {
        float za, zb;
        box_muller2(orc_uniform_f32(wa[2]), orc_uniform_f32(wa[3]), &za, &zb);
        a += (int)lrintf(read_noise * za);
        b += (int)lrintf(read_noise * zb);
    }
    *na = a;
    *nb = b;
}

/* ------------------------------------------------------------------------------------------ */
/* Reduced-precision reconstructor (NEXT variant f1): the number formats, written from their     */
/* definitions                                                                                  */
/* ------------------------------------------------------------------------------------------ */

/* bfloat16 = the upper 16 bits of an IEEE binary32 (1 sign, 8 exponent, 7 fraction bits); from
 * float by round to nearest, ties to even.  Inputs are finite. */
uint16_t orc_bf16_rn(float x) {
    uint32_t u = bits_from_f32(x);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float orc_bf16_to_f32(uint16_t h) { return f32_from_bits((uint32_t)h << 16); }

/* FP8 E4M3 in the OCP 8-bit floating-point format ("E4M3FN"): 1 sign, 4 exponent (bias 7) and 3
 * fraction bits, subnormals below 2^-6 with step 2^-9, no infinities, S.1111.111 is NaN, so the
 * largest finite magnitude is 1.75 * 2^8 = 448.  From float by round to nearest, ties to even,
 * saturating to +-448. */
uint8_t orc_e4m3_rn_sat(float x) {
    if (x != x) return 0x7f;
    uint8_t sgn = signbit(x) ? 0x80 : 0x00;
    double a = fabs((double)x);
    if (a >= 448.0) return sgn | 0x7e;
    if (a < ldexp(1.0, -6)) return sgn | (uint8_t)nearbyint(a * 512.0);   /* m * 2^-9, m <= 8 */
    int e;
    double f = frexp(a, &e);             /* a = f 2^e, f in [1/2, 1) */
    int E = e - 1;
    double m = nearbyint((2.0 * f - 1.0) * 8.0);
    if (m == 8.0) { m = 0.0; E += 1; }
    int code = ((E + 7) << 3) | (int)m;
    if (code > 0x7e) code = 0x7e;
    return sgn | (uint8_t)code;
}
float orc_e4m3_to_f32(uint8_t b) {
    int e = (b >> 3) & 15, m = b & 7;
    double v;
    if (e == 15 && m == 7) v = NAN;
    else if (e == 0) v = ldexp((double)m, -9);
    else v = ldexp(1.0 + m / 8.0, e - 7);
    return (float)((b & 0x80) ? -v : v);
}

/* Quantize rows of R [rows][cols] (row stride ld).  dtype 1: bfloat16 codes, scale 1.
 * dtype 2: scale_r = fl(max_j |R_rj| / 448) (1 for an all-zero row), codes e4m3(fl(R_rj / scale_r)).
 * The represented value is code value * scale_r. */
void orc_quantize_rows(const float* R, int rows, int cols, int ld, int dtype, void* out, float* scales) {
    for (int r = 0; r < rows; ++r) {
        const float* row = R + (size_t)r * ld;
        if (dtype == 1) {
            uint16_t* o = (uint16_t*)out + (size_t)r * cols;
            for (int j = 0; j < cols; ++j) o[j] = orc_bf16_rn(row[j]);
            if (scales) scales[r] = 1.0f;
        } else {
            uint8_t* o = (uint8_t*)out + (size_t)r * cols;
            float amax = 0.0f;
            for (int j = 0; j < cols; ++j) amax = fmaxf(amax, fabsf(row[j]));
            /* a scale below the smallest normal float (2^-126; also 0 when the row is zero or
             * max / 448 underflows) is replaced by 1: the row's entries are then all below
             * 448 2^-126 and encode to zero, instead of 0 / 0 codes */
            float sc = amax / 448.0f;
            if (!(sc >= FLT_MIN)) sc = 1.0f;
            for (int j = 0; j < cols; ++j) o[j] = orc_e4m3_rn_sat(row[j] / sc);
            if (scales) scales[r] = sc;
        }
    }
}

/* Noisy frame of n pixels for counters (pixel0 + i, step, wfs). */
/* Noisy frames of n pixels in subaperture frames of frame_px pixels each (pixel i of the buffer
 * has frame index pixel0 + i; pairs within each frame). */
void orc_noise_frame(const float* lam, int n, int frame_px, float read_noise, uint32_t pixel0, uint32_t step,
                     uint32_t wfs, uint64_t seed, int32_t* out) {
    const int half = frame_px / 2;
    for (int f = 0; f + frame_px <= n; f += frame_px)
        for (int q = 0; q < half; ++q)
            orc_noise_pair(lam[f + q], lam[f + q + half], read_noise, pixel0 + (uint32_t)(f + q), step, wfs, seed,
                           &out[f + q], &out[f + q + half]);
}

/* ------------------------------------------------------------------------------------------ */
/* simulation state                                                                           */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    orc_wfs p;
    int N;                    /* pupil samples across D = n_sub n_px                            */
    double dx;                /* pupil sample pitch, m                                           */
    int n_det, n_valid;
    double* A;                /* [N][N] amplitude                                               */
    int* valid_idx;           /* [n_valid] subaperture index sy*n_sub+sx, row-major order       */
    double* frac;             /* [n_valid] illuminated fraction                                 */
    double* sigma_pix;        /* [n_valid] elongation sigma in image pixels (0 = none)          */
    double* dir;              /* [n_valid][2] elongation direction                              */
    int slope0;               /* offset of this WFS in the slope vector                         */
    orc_plan* plan;
    float* lam;               /* [n_valid][n_det^2] last intensities (float) when recorded      */
    int32_t* frames;          /* [n_valid][n_det^2] last noisy frames                           */
} wfs_state;

typedef struct {
    orc_sci p;
    int N, M;                 /* pupil samples, FFT size M = pad N                              */
    double dx, sumA;
    double* A;
    double* psf;              /* [M][M] accumulated, fftshifted                                  */
    orc_plan* plan;
    double sr_sum, sr_last;
    double var_sum, var_last;   /* Marechal: residual phase variance per step (science band)    */
    long n_psf, n_sr;
} sci_state;

typedef struct {
    orc_config cfg;
    int n_wfs, n_sci, n_layers, n_dms;
    orc_wfs* wfs_p; orc_sci* sci_p; orc_layer* lay_p; orc_dm* dm_p;
    wfs_state* wfs;
    sci_state* sci;
    double** screen;          /* promoted layers                                                 */
    double** surf;            /* DM surfaces [surf_n][surf_n]                                    */
    int* dm_nvalid; int* dm_cmd0;
    double* misreg;           /* [n_dms][4]: shift_x, shift_y (m), rotation (rad), magnification */
    int n_cmd, n_slopes;
    const float* R; double* s_ref;
    int r_dtype;
    uint16_t* Rb;             /* bfloat16 codes of R (r_dtype 1)                                 */
    uint8_t* Rq;              /* E4M3 codes of R (r_dtype 2)                                     */
    float* r_scale;           /* per-row scales (r_dtype 2)                                      */
    double* c;                /* commands                                                        */
    double* c_prev;           /* commands of the previous step (second-order controller)         */
    double* dc_prev;          /* reconstructed update of the previous step                       */
    double ctl[4];            /* controller a1, a2, b0, b1; NaN a1 = pure integrator of gain g   */
    double* s;                /* last slopes                                                     */
    long k;                   /* step counter                                                    */
    int record;               /* keep float intensities / frames                                 */
} orc_sim;

static void sim_free(orc_sim* S);

/* Elongation of every valid subaperture of a laser star: the spot seen from a subaperture at
 * distance b from the launch spans b dh / H^2 rad (FWHM) along the launch-to-subaperture
 * direction (dh the sodium layer thickness, H its height). */
static void set_elongation(wfs_state* W) {
    for (int v = 0; v < W->n_valid; ++v) {
        W->sigma_pix[v] = 0.0;
        W->dir[2 * v] = W->dir[2 * v + 1] = 0.0;
    }
    if (!(W->p.type == 1 && W->p.na_fwhm > 0.0)) return;
    double pix_rad = W->p.lambda / ((double)W->p.n_fft * W->dx);
    for (int v = 0; v < W->n_valid; ++v) {
        int sx = W->valid_idx[v] % W->p.n_sub, sy = W->valid_idx[v] / W->p.n_sub;
        double cx = ((double)sx - 0.5 * (double)(W->p.n_sub - 1)) * W->p.n_px * W->dx - W->p.launch_x;
        double cy = ((double)sy - 0.5 * (double)(W->p.n_sub - 1)) * W->p.n_px * W->dx - W->p.launch_y;
        double b = sqrt(cx * cx + cy * cy);
        if (b > 0.0) {
            double fwhm = b * W->p.na_fwhm / (W->p.height * W->p.height);
            W->sigma_pix[v] = fwhm / (2.0 * sqrt(2.0 * log(2.0))) / pix_rad;
            W->dir[2 * v] = cx / b; W->dir[2 * v + 1] = cy / b;
        }
    }
}

/* Sodium layer evolution ("The closed loop": the sodium layer temporal evolution may be
 * considered): new height (cone projection of the laser star) and thickness (elongation) of
 * the layer seen by laser sensor w, from the next step on.  Returns 0, or -1 for a sensor that
 * is not a laser star or a height not above every layer. */
int orc_set_sodium(orc_sim* S, int w, double height, double na_fwhm) {
    if (w < 0 || w >= S->n_wfs || S->wfs[w].p.type != 1 || !(height > 0.0) || !(na_fwhm >= 0.0)) return -1;
    for (int l = 0; l < S->n_layers; ++l)
        if (S->lay_p[l].alt >= height) return -1;
    S->wfs[w].p.height = height;
    S->wfs[w].p.na_fwhm = na_fwhm;
    set_elongation(&S->wfs[w]);
    return 0;
}

/* Phase (rad at the reference wavelength) along a direction: layers minus DM surfaces at the
 * cone-beam projection x (1 - h/H) + h theta (H infinite for natural stars), plus the
 * frozen-flow offset (k dt) v for layers.  x, y in metres in the pupil. */
static double residual_phase(const orc_sim* S, double x, double y, double thx, double thy,
                             double H, double t) {
    double phi = 0.0;
    for (int l = 0; l < S->n_layers; ++l) {
        const orc_layer* L = &S->lay_p[l];
        double f = (H > 0.0) ? 1.0 - L->alt / H : 1.0;
        double u = x * f + L->alt * thx + t * L->vx;
        double v = y * f + L->alt * thy + t * L->vy;
        double fx = u / L->pixel + 0.5 * (double)(L->n - 1);
        double fy = v / L->pixel + 0.5 * (double)(L->n - 1);
        phi += orc_bilinear_periodic(S->screen[l], L->n, fx, fy);
    }
    for (int m = 0; m < S->n_dms; ++m) {
        const orc_dm* M = &S->dm_p[m];
        double f = (H > 0.0) ? 1.0 - M->alt / H : 1.0;
        double u = x * f + M->alt * thx;
        double v = y * f + M->alt * thy;
        double fx = u / M->surf_dx + 0.5 * (double)(M->surf_n - 1);
        double fy = v / M->surf_dx + 0.5 * (double)(M->surf_n - 1);
        phi -= orc_bilinear_clamped(S->surf[m], M->surf_n, fx, fy);
    }
    return phi;
}

static void update_dm_surfaces(orc_sim* S) {
    for (int m = 0; m < S->n_dms; ++m) {
        const orc_dm* M = &S->dm_p[m];
        double* C = (double*)calloc((size_t)M->nx * M->ny, sizeof(double));
        int q = S->dm_cmd0[m];
        for (int a = 0; a < M->nx * M->ny; ++a)
            if (M->valid[a]) C[a] = S->c[q++];
        const double* T = &S->misreg[4 * m];
        if (T[0] == 0.0 && T[1] == 0.0 && T[2] == 0.0 && T[3] == 1.0)
            orc_dm_surface(M->nx, M->ny, M->pitch, M->coupling, M->surf_n, M->surf_dx, C, S->surf[m]);
        else
            orc_dm_surface_misreg(M->nx, M->ny, M->pitch, M->coupling, M->surf_n, M->surf_dx, T[0], T[1], T[2],
                                  T[3], C, S->surf[m]);
        free(C);
    }
}

orc_sim* orc_create(const orc_config* cfg) {
    orc_sim* S = (orc_sim*)calloc(1, sizeof(orc_sim));
    S->cfg = *cfg;
    S->n_wfs = cfg->n_wfs; S->n_sci = cfg->n_sci; S->n_layers = cfg->n_layers; S->n_dms = cfg->n_dms;
    S->wfs_p = (orc_wfs*)malloc(sizeof(orc_wfs) * (S->n_wfs ? S->n_wfs : 1));
    S->sci_p = (orc_sci*)malloc(sizeof(orc_sci) * (S->n_sci ? S->n_sci : 1));
    S->lay_p = (orc_layer*)malloc(sizeof(orc_layer) * (S->n_layers ? S->n_layers : 1));
    S->dm_p = (orc_dm*)malloc(sizeof(orc_dm) * (S->n_dms ? S->n_dms : 1));
    memcpy(S->wfs_p, cfg->wfs, sizeof(orc_wfs) * S->n_wfs);
    memcpy(S->sci_p, cfg->sci, sizeof(orc_sci) * S->n_sci);
    memcpy(S->lay_p, cfg->layers, sizeof(orc_layer) * S->n_layers);
    memcpy(S->dm_p, cfg->dms, sizeof(orc_dm) * S->n_dms);

    S->screen = (double**)calloc(S->n_layers ? S->n_layers : 1, sizeof(double*));
    for (int l = 0; l < S->n_layers; ++l) {
        size_t n2 = (size_t)S->lay_p[l].n * S->lay_p[l].n;
        S->screen[l] = (double*)malloc(sizeof(double) * n2);
        for (size_t q = 0; q < n2; ++q) S->screen[l][q] = (double)cfg->layers[l].phase[q];
        S->lay_p[l].phase = NULL;
    }
    S->surf = (double**)calloc(S->n_dms ? S->n_dms : 1, sizeof(double*));
    S->dm_nvalid = (int*)calloc(S->n_dms ? S->n_dms : 1, sizeof(int));
    S->dm_cmd0 = (int*)calloc(S->n_dms ? S->n_dms : 1, sizeof(int));
    S->misreg = (double*)calloc(4 * (size_t)(S->n_dms ? S->n_dms : 1), sizeof(double));
    for (int m = 0; m < S->n_dms; ++m) S->misreg[4 * m + 3] = 1.0;
    int ncmd = 0;
    for (int m = 0; m < S->n_dms; ++m) {
        orc_dm* M = &S->dm_p[m];
        uint8_t* v = (uint8_t*)malloc((size_t)M->nx * M->ny);
        memcpy(v, cfg->dms[m].valid, (size_t)M->nx * M->ny);
        M->valid = v;
        int cnt = 0;
        for (int a = 0; a < M->nx * M->ny; ++a) cnt += v[a] ? 1 : 0;
        S->dm_nvalid[m] = cnt; S->dm_cmd0[m] = ncmd; ncmd += cnt;
        S->surf[m] = (double*)calloc((size_t)M->surf_n * M->surf_n, sizeof(double));
    }
    S->n_cmd = ncmd;

    S->wfs = (wfs_state*)calloc(S->n_wfs ? S->n_wfs : 1, sizeof(wfs_state));
    int ns = 0;
    for (int w = 0; w < S->n_wfs; ++w) {
        wfs_state* W = &S->wfs[w];
        W->p = S->wfs_p[w];
        W->N = W->p.n_sub * W->p.n_px;
        W->dx = cfg->D / (double)W->N;
        W->n_det = W->p.n_fft / W->p.n_bin;
        W->A = (double*)malloc(sizeof(double) * (size_t)W->N * W->N);
        orc_pupil(cfg->D, cfg->obstruction, W->N, W->A);
        int nsub2 = W->p.n_sub * W->p.n_sub;
        int* vmap = (int*)malloc(sizeof(int) * nsub2);
        double* fr = (double*)malloc(sizeof(double) * nsub2);
        W->n_valid = orc_valid_subaps(W->A, W->p.n_sub, W->p.n_px, W->p.valid_thr, vmap, fr);
        W->valid_idx = (int*)malloc(sizeof(int) * (W->n_valid ? W->n_valid : 1));
        W->frac = (double*)malloc(sizeof(double) * (W->n_valid ? W->n_valid : 1));
        W->sigma_pix = (double*)calloc(W->n_valid ? W->n_valid : 1, sizeof(double));
        W->dir = (double*)calloc(2 * (W->n_valid ? W->n_valid : 1), sizeof(double));
        int q = 0;
        for (int i = 0; i < nsub2; ++i)
            if (vmap[i]) { W->valid_idx[q] = i; W->frac[q] = fr[i]; ++q; }
        free(vmap); free(fr);
        set_elongation(W);
        W->slope0 = ns;
        ns += 2 * W->n_valid;
        W->plan = plan_new(W->p.n_fft);
        W->lam = (float*)calloc((size_t)(W->n_valid ? W->n_valid : 1) * W->n_det * W->n_det, sizeof(float));
        W->frames = (int32_t*)calloc((size_t)(W->n_valid ? W->n_valid : 1) * W->n_det * W->n_det, sizeof(int32_t));
    }
    S->n_slopes = ns;
    if ((cfg->R && (cfg->n_cmd != S->n_cmd || cfg->n_slopes != S->n_slopes))) { sim_free(S); return NULL; }
    S->R = cfg->R;
    S->r_dtype = cfg->r_dtype;
    if (S->R && S->r_dtype == 1) {
        S->Rb = (uint16_t*)malloc(sizeof(uint16_t) * (size_t)S->n_cmd * ns);
        orc_quantize_rows(S->R, S->n_cmd, ns, ns, 1, S->Rb, NULL);
    } else if (S->R && S->r_dtype == 2) {
        S->Rq = (uint8_t*)malloc((size_t)S->n_cmd * ns);
        S->r_scale = (float*)malloc(sizeof(float) * (S->n_cmd ? S->n_cmd : 1));
        orc_quantize_rows(S->R, S->n_cmd, ns, ns, 2, S->Rq, S->r_scale);
    }
    S->s_ref = (double*)calloc(ns ? ns : 1, sizeof(double));
    if (cfg->s_ref) for (int i = 0; i < ns; ++i) S->s_ref[i] = (double)cfg->s_ref[i];
    S->c = (double*)calloc(S->n_cmd ? S->n_cmd : 1, sizeof(double));
    S->c_prev = (double*)calloc(S->n_cmd ? S->n_cmd : 1, sizeof(double));
    S->dc_prev = (double*)calloc(S->n_cmd ? S->n_cmd : 1, sizeof(double));
    S->ctl[0] = NAN;
    S->s = (double*)calloc(ns ? ns : 1, sizeof(double));

    S->sci = (sci_state*)calloc(S->n_sci ? S->n_sci : 1, sizeof(sci_state));
    for (int q = 0; q < S->n_sci; ++q) {
        sci_state* C = &S->sci[q];
        C->p = S->sci_p[q];
        C->N = C->p.n_px; C->M = C->p.n_px * C->p.pad;
        C->dx = cfg->D / (double)C->N;
        C->A = (double*)malloc(sizeof(double) * (size_t)C->N * C->N);
        orc_pupil(cfg->D, cfg->obstruction, C->N, C->A);
        C->sumA = 0.0;
        for (size_t i = 0; i < (size_t)C->N * C->N; ++i) C->sumA += C->A[i];
        C->psf = (double*)calloc((size_t)C->M * C->M, sizeof(double));
        C->plan = plan_new(C->M);
    }
    S->record = 1;
    return S;
}

static void sim_free(orc_sim* S) {
    if (!S) return;
    for (int l = 0; l < S->n_layers; ++l) free(S->screen[l]);
    for (int m = 0; m < S->n_dms; ++m) { free(S->surf[m]); free((void*)S->dm_p[m].valid); }
    for (int w = 0; w < S->n_wfs; ++w) {
        wfs_state* W = &S->wfs[w];
        free(W->A); free(W->valid_idx); free(W->frac); free(W->sigma_pix); free(W->dir);
        plan_free(W->plan); free(W->lam); free(W->frames);
    }
    for (int q = 0; q < S->n_sci; ++q) { free(S->sci[q].A); free(S->sci[q].psf); plan_free(S->sci[q].plan); }
    free(S->screen); free(S->surf); free(S->dm_nvalid); free(S->dm_cmd0); free(S->misreg);
    free(S->wfs); free(S->sci); free(S->wfs_p); free(S->sci_p); free(S->lay_p); free(S->dm_p);
    free(S->s_ref); free(S->c); free(S->s); free(S->c_prev); free(S->dc_prev);
    free(S->Rb); free(S->Rq); free(S->r_scale);
    free(S);
}
void orc_destroy(orc_sim* S) { sim_free(S); }

/* Residual phase (rad at the reference wavelength) of WFS w on its full pupil grid at the
 * current step and commands; DM surfaces are refreshed from the commands first. */
void orc_wfs_phase(orc_sim* S, int w, double* out) {
    update_dm_surfaces(S);
    wfs_state* W = &S->wfs[w];
    double H = W->p.type == 1 ? W->p.height : 0.0, t = (double)S->k * S->cfg.dt;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < W->N; ++j)
        for (int i = 0; i < W->N; ++i) {
            double x = ((double)i - 0.5 * (double)(W->N - 1)) * W->dx;
            double y = ((double)j - 0.5 * (double)(W->N - 1)) * W->dx;
            out[(size_t)j * W->N + i] = residual_phase(S, x, y, W->p.theta_x, W->p.theta_y, H, t);
        }
}

/* Slopes of every WFS at the current step and commands (a3-a9), written to S->s. */
static void measure_slopes(orc_sim* S) {
    double t = (double)S->k * S->cfg.dt;
    for (int w = 0; w < S->n_wfs; ++w) {
        wfs_state* W = &S->wfs[w];
        double H = W->p.type == 1 ? W->p.height : 0.0;
        double scale = S->cfg.lambda_ref / W->p.lambda;
        int npx = W->p.n_px, N = W->p.n_fft, nd = W->n_det;
        #pragma omp parallel for schedule(dynamic, 4)
        for (int v = 0; v < W->n_valid; ++v) {
            double* amp = (double*)malloc(sizeof(double) * npx * npx);
            double* ph = (double*)malloc(sizeof(double) * npx * npx);
            double* img = (double*)malloc(sizeof(double) * (size_t)N * N);
            double* work = (double*)malloc(sizeof(double) * ((size_t)2 * N * N + 6 * N));
            double* det = (double*)malloc(sizeof(double) * nd * nd);
            int sx = W->valid_idx[v] % W->p.n_sub, sy = W->valid_idx[v] / W->p.n_sub;
            for (int y = 0; y < npx; ++y)
                for (int x = 0; x < npx; ++x) {
                    int i = sx * npx + x, j = sy * npx + y;
                    double px = ((double)i - 0.5 * (double)(W->N - 1)) * W->dx;
                    double py = ((double)j - 0.5 * (double)(W->N - 1)) * W->dx;
                    amp[y * npx + x] = W->A[(size_t)j * W->N + i];
                    ph[y * npx + x] = scale * residual_phase(S, px, py, W->p.theta_x, W->p.theta_y, H, t);
                }
            sh_image_plan(npx, W->plan, amp, ph, W->sigma_pix[v], W->dir[2 * v], W->dir[2 * v + 1], img, work);
            orc_bin(N, W->p.n_bin, img, det);
            double tot = 0.0;
            for (int q = 0; q < nd * nd; ++q) tot += det[q];
            double norm = W->p.n_photons * W->frac[v] / tot;
            for (int q = 0; q < nd * nd; ++q) det[q] *= norm;
            size_t base = (size_t)v * nd * nd;
            for (int q = 0; q < nd * nd; ++q) W->lam[base + q] = (float)det[q];
            if (S->cfg.noise) {
                const int half = nd * nd / 2;
                for (int q = 0; q < half; ++q) {
                    orc_noise_pair(W->lam[base + q], W->lam[base + q + half], (float)W->p.read_noise,
                                   (uint32_t)(base + q), (uint32_t)S->k, (uint32_t)w, S->cfg.seed,
                                   &W->frames[base + q], &W->frames[base + q + half]);
                    det[q] = (double)W->frames[base + q];
                    det[q + half] = (double)W->frames[base + q + half];
                }
            }
            double gx, gy;
            orc_cog(nd, det, &gx, &gy);
            S->s[W->slope0 + v] = gx - S->s_ref[W->slope0 + v];
            S->s[W->slope0 + W->n_valid + v] = gy - S->s_ref[W->slope0 + W->n_valid + v];
            free(amp); free(ph); free(img); free(work); free(det);
        }
    }
}

/* Science direction q at the current step: instantaneous Strehl and the PSF increment. */
static void science_step(orc_sim* S, int q, int do_psf) {
    sci_state* C = &S->sci[q];
    double t = (double)S->k * S->cfg.dt, scale = S->cfg.lambda_ref / C->p.lambda;
    int N = C->N, M = C->M;
    double* er = (double*)calloc((size_t)M * M, sizeof(double));
    double* ei = (double*)calloc((size_t)M * M, sizeof(double));
    double* pw = (double*)calloc((size_t)N * N, sizeof(double));   /* science-band phase */
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            double x = ((double)i - 0.5 * (double)(N - 1)) * C->dx;
            double y = ((double)j - 0.5 * (double)(N - 1)) * C->dx;
            double a = C->A[(size_t)j * N + i];
            double ph = scale * residual_phase(S, x, y, C->p.theta_x, C->p.theta_y, 0.0, t);
            pw[(size_t)j * N + i] = ph;
            er[(size_t)j * M + i] = a * cos(ph);
            ei[(size_t)j * M + i] = a * sin(ph);
        }
    double fr = 0.0, fi = 0.0, s1 = 0.0, s2 = 0.0;
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            fr += er[(size_t)j * M + i];
            fi += ei[(size_t)j * M + i];
            double a = C->A[(size_t)j * N + i], ph = pw[(size_t)j * N + i];
            s1 += a * ph;
            s2 += a * ph * ph;
        }
    free(pw);
    C->sr_last = (fr * fr + fi * fi) / (C->sumA * C->sumA);
    C->sr_sum += C->sr_last;
    C->n_sr += 1;
    /* Marechal ("Strehl Ratio on the closed-loop wavefront history"): piston-removed,
     * amplitude-weighted phase variance over the pupil at the science wavelength */
    double mean = s1 / C->sumA;
    C->var_last = s2 / C->sumA - mean * mean;
    C->var_sum += C->var_last;
    if (do_psf) {
        /* 2-D FFT: rows in parallel, then columns in parallel */
        #pragma omp parallel
        {
            double* ws = (double*)malloc(sizeof(double) * 6 * M);
            double* cr = (double*)malloc(sizeof(double) * M);
            double* ci = (double*)malloc(sizeof(double) * M);
            #pragma omp for schedule(static)
            for (int y = 0; y < M; ++y) fft1_plan(C->plan, er + (size_t)y * M, ei + (size_t)y * M, 0, ws);
            #pragma omp for schedule(static)
            for (int x = 0; x < M; ++x) {
                for (int y = 0; y < M; ++y) { cr[y] = er[(size_t)y * M + x]; ci[y] = ei[(size_t)y * M + x]; }
                fft1_plan(C->plan, cr, ci, 0, ws);
                for (int y = 0; y < M; ++y) { er[(size_t)y * M + x] = cr[y]; ei[(size_t)y * M + x] = ci[y]; }
            }
            free(ws); free(cr); free(ci);
        }
        for (int j = 0; j < M; ++j)
            for (int i = 0; i < M; ++i) {
                size_t src = (size_t)((j + M / 2) % M) * M + (i + M / 2) % M;
                C->psf[(size_t)j * M + i] += er[src] * er[src] + ei[src] * ei[src];
            }
        C->n_psf += 1;
    }
    free(er); free(ei);
}

/* One closed-loop step: DM surfaces from c_k, slopes s_k, science at step k, then
 * c_{k+1} = c_k + g R s_k (one frame of delay), k <- k + 1. */
int orc_step(orc_sim* S, int n_steps) {
    if (!S->R && S->n_cmd > 0 && S->n_slopes > 0) return -1;
    for (int it = 0; it < n_steps; ++it) {
        update_dm_surfaces(S);
        measure_slopes(S);
        int do_psf = S->cfg.psf_every > 0 && (S->k % S->cfg.psf_every) == 0;
        for (int q = 0; q < S->n_sci; ++q) science_step(S, q, do_psf);
        double* dc = (double*)malloc(sizeof(double) * (S->n_cmd ? S->n_cmd : 1));
        #pragma omp parallel for schedule(static)
        for (int i = 0; i < S->n_cmd; ++i) {
            double acc = 0.0;
            if (S->r_dtype == 1) {
                const uint16_t* row = S->Rb + (size_t)i * S->n_slopes;
                for (int j = 0; j < S->n_slopes; ++j) acc += (double)orc_bf16_to_f32(row[j]) * S->s[j];
            } else if (S->r_dtype == 2) {
                const uint8_t* row = S->Rq + (size_t)i * S->n_slopes;
                const double sc = (double)S->r_scale[i];
                for (int j = 0; j < S->n_slopes; ++j) acc += (double)orc_e4m3_to_f32(row[j]) * sc * S->s[j];
            } else {
                const float* row = S->R + (size_t)i * S->n_slopes;
                for (int j = 0; j < S->n_slopes; ++j) acc += (double)row[j] * S->s[j];
            }
            dc[i] = acc;
        }
        if (isnan(S->ctl[0])) {
            for (int i = 0; i < S->n_cmd; ++i) S->c[i] += S->cfg.gain * dc[i];
        } else {
            /* second-order controller ("The closed loop": a pure integrator or a second-order
             * low-pass filter), read as the recursion per command
             * c_{k+1} = a1 c_k + a2 c_{k-1} + b0 dc_k + b1 dc_{k-1} */
            for (int i = 0; i < S->n_cmd; ++i) {
                double cn = S->ctl[0] * S->c[i] + S->ctl[1] * S->c_prev[i] + S->ctl[2] * dc[i] + S->ctl[3] * S->dc_prev[i];
                S->c_prev[i] = S->c[i];
                S->dc_prev[i] = dc[i];
                S->c[i] = cn;
            }
        }
        free(dc);
        S->k += 1;
    }
    return 0;
}

/* Slopes at the current state without advancing time or touching the commands (used to
 * calibrate interaction matrices by pokes). */
void orc_measure(orc_sim* S, double* out) {
    update_dm_surfaces(S);
    measure_slopes(S);
    memcpy(out, S->s, sizeof(double) * S->n_slopes);
}

int orc_n_cmd(const orc_sim* S) { return S->n_cmd; }
int orc_n_slopes(const orc_sim* S) { return S->n_slopes; }
int orc_n_valid(const orc_sim* S, int w) { return S->wfs[w].n_valid; }
long orc_step_index(const orc_sim* S) { return S->k; }
void orc_set_step_index(orc_sim* S, long k) { S->k = k; }
/* Marechal Strehl of science direction q: exp(-mean over steps of the residual variance) and
 * exp(-variance) of the last step. */
void orc_marechal(const orc_sim* S, int q, double* sr_long, double* sr_last) {
    const sci_state* C = &S->sci[q];
    *sr_long = C->n_sr ? exp(-C->var_sum / (double)C->n_sr) : 0.0;
    *sr_last = exp(-C->var_last);
}
void orc_get_valid(const orc_sim* S, int w, int* idx) {
    memcpy(idx, S->wfs[w].valid_idx, sizeof(int) * S->wfs[w].n_valid);
}
/* Misregistration of DM m (shift in m at its conjugate altitude, rotation in rad, magnification)
 * from the next measurement or step on.  Returns -1 for a bad index or magnification <= 0. */
int orc_set_misregistration(orc_sim* S, int m, double shift_x, double shift_y, double rot, double mag) {
    if (m < 0 || m >= S->n_dms || !(mag > 0.0)) return -1;
    double* T = &S->misreg[4 * m];
    T[0] = shift_x; T[1] = shift_y; T[2] = rot; T[3] = mag;
    return 0;
}

/* Elongation of sensor w's valid subapertures: sigma in image pixels and unit direction. */
void orc_get_elongation(const orc_sim* S, int w, double* sigma_pix, double* dir) {
    memcpy(sigma_pix, S->wfs[w].sigma_pix, sizeof(double) * S->wfs[w].n_valid);
    memcpy(dir, S->wfs[w].dir, sizeof(double) * 2 * S->wfs[w].n_valid);
}
void orc_get_slopes(const orc_sim* S, double* out) { memcpy(out, S->s, sizeof(double) * S->n_slopes); }
void orc_get_commands(const orc_sim* S, double* out) { memcpy(out, S->c, sizeof(double) * S->n_cmd); }
void orc_set_commands(orc_sim* S, const double* in) {
    memcpy(S->c, in, sizeof(double) * S->n_cmd);
    memcpy(S->c_prev, in, sizeof(double) * S->n_cmd);
    memset(S->dc_prev, 0, sizeof(double) * S->n_cmd);
}
/* Second-order controller coefficients (a1, a2, b0, b1); the filter's memory starts from the
 * current commands and a zero update. */
void orc_set_controller(orc_sim* S, double a1, double a2, double b0, double b1) {
    S->ctl[0] = a1; S->ctl[1] = a2; S->ctl[2] = b0; S->ctl[3] = b1;
    memcpy(S->c_prev, S->c, sizeof(double) * S->n_cmd);
    memset(S->dc_prev, 0, sizeof(double) * S->n_cmd);
}
void orc_get_dm_surface(orc_sim* S, int m, double* out) {
    update_dm_surfaces(S);
    size_t n = (size_t)S->dm_p[m].surf_n;
    memcpy(out, S->surf[m], sizeof(double) * n * n);
}
void orc_get_frames(const orc_sim* S, int w, float* lam, int32_t* frames) {
    const wfs_state* W = &S->wfs[w];
    size_t n = (size_t)W->n_valid * W->n_det * W->n_det;
    if (lam) memcpy(lam, W->lam, sizeof(float) * n);
    if (frames) memcpy(frames, W->frames, sizeof(int32_t) * n);
}
/* PSF normalised by the diffraction-limited peak (sum A)^2 per accumulated frame; long-exposure
 * Strehl = mean of the instantaneous on-axis Strehl values. */
void orc_get_psf(const orc_sim* S, int q, double* out, double* sr_long, double* sr_last) {
    const sci_state* C = &S->sci[q];
    size_t n = (size_t)C->M * C->M;
    double norm = (C->n_psf > 0) ? 1.0 / ((double)C->n_psf * C->sumA * C->sumA) : 0.0;
    if (out) for (size_t i = 0; i < n; ++i) out[i] = C->psf[i] * norm;
    if (sr_long) *sr_long = C->n_sr ? C->sr_sum / (double)C->n_sr : 0.0;
    if (sr_last) *sr_last = C->sr_last;
}
int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
