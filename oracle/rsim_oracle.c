/*
 * rsim_oracle.c -- plain, slow FP64 CPU oracle of the coherent scatterer -> IQ
 * summation of arXiv 2408.11472 ("High Performance Simulation of Spaceborne
 * Radar for Remote-Sensing Oceanography"), regular mode and fast mode.
 *
 * TEST INFRASTRUCTURE ONLY.  It is called by the test-suite, by the smoke check
 * and by the benchmark's CPU-baseline leg, never by the library's product path.
 * It shares no code, header, table or constant with the CUDA implementation.
 *
 * Everything is computed in IEEE double from the same float32 input arrays the
 * GPU reads (promoted exactly to double).  Parallelism: OpenMP over a FIXED
 * number of scatterer chunks (independent of the thread count); chunk partial
 * sums are Neumaier-compensated and merged in chunk order, so the result does
 * not depend on how many threads ran.
 *
 * Definitions (paper section / equation, and the reading taken where the paper
 * is silent):
 *   t_p      = p / PRF                                   (stop-and-hop)
 *   s(t)     = O + r + v (t - t0),  P(t) = p0 + V t,  d = P - s   (Alg. 1 update_simulation, linear
 *              kinematics from the state given at epoch t0)
 *   R        = |d|,  dR = R - r_ref(t)  (evaluated without cancellation, see echo_at)
 *   theta    = atan2(|d_xy|, d_z)                          (nadir-pointing antenna)
 *   w        = exp(-2 ln2 theta^2/theta_b^2)               (analytic two-way pattern), or
 *            = the complex two-way pattern G(u, v) tabulated on a u-v grid and interpolated
 *              bilinearly (real and imaginary parts) at the facet's direction cosines
 *              u = (s - P)_x / R, v = (s - P)_y / R; zero outside the grid (Sec. II.A)
 *   C        = sqrt(sigma A) w (r_ref/R)^2 exp(-j 2 pi (psi - rint psi)),  psi = 2 R / lambda
 *              [cycles]                                   (radar equation at facet level, Sec. II.A)
 *   gate     = floor(dR / gate_width + N_g / 2), kept iff 0 <= gate < N_g  (complex sum per range gate, Sec. II.A)
 *   regular  : Y[p, g] = sum_n C_n(t_p) [gate_n(t_p) = g]                (Fig. 1 step 4)
 *   fast     : for each update i (pulse p_i = i n_fast), Algorithm 1:
 *                C_i, R_i at t(p_i);  C_{i+1} at t(p_i + 1);
 *                D_i = arg(conj(C_{i+1}) C_i) PRF              [rad/s]
 *                nu  = -D_i / (2 pi PRF)                      [cycles/pulse, in [-1/2, 1/2)]
 *                      (the phase change of C over the pair, its geometric part taken
 *                      from the range change R_{i+1} - R_i written without cancellation)
 *                bin = floor(nu N_d + 1/2) mod N_d            (nearest DFT bin)
 *                T[i, gate(R_i), bin] += C_i                  (rasterize)
 *              then post-processing (Sec. III.B): unnormalised inverse DFT along
 *              the Doppler axis, s_i[g, m] = sum_k T[i,g,k] exp(+j 2 pi k m / N_d),
 *              Eq. (1) weights W_i(x) on |p_i - x| / n_fast, and
 *              Y[x, g] = sum_i W_i(x) s_i[g, (x - p_i) mod N_d].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_NCHUNK 64
#define OR_PI 3.14159265358979323846
#define OR_LN2 0.69314718055994530942

typedef struct {
    double carrier_hz, prf_hz, c_mps, gate_width_m, beamwidth_rad;
    int32_t n_gates;
    int32_t ant_nu;      /* > 0: tabulated pattern with ant_nu x ant_nv nodes */
    const double *ant;   /* [ant_nv][ant_nu][2] complex two-way gain, or NULL */
    int32_t ant_nv;
    int32_t pad_;
    double ant_u0, ant_du, ant_v0, ant_dv;
} or_radar;

typedef struct {
    double p0[3], v[3];
    double r_ref0, r_ref_rate;
} or_platform;

typedef struct {
    int64_t n;
    const float *x, *y, *z, *vx, *vy, *vz, *nrcs;
    double origin[3];
    double area;
    double t0;   /* epoch of the state: s(t) = O + r + v (t - t0) */
} or_scene;

typedef struct {
    double R, dR, rho, dx, dy, dz, theta, amp, psi, re, im;
    double g_re, g_im;   /* complex two-way gain G of the pattern (the Gaussian pattern: real) */
    /* tabulated pattern only: base = sqrt(sigma A) (r_ref/R)^2, phase factor (cr, ci),
     * direction cosines (u, v) and dG/du, dG/dv (complex) */
    double base, cr, ci, u, v, gu_re, gu_im, gv_re, gv_im;
} or_echo;

/* Bilinear interpolation of the tabulated complex pattern at (u, v): nodes at
 * u0 + i du (i < nu), v0 + j dv (j < nv); the cell (i, j) holds u0 + i du <= u < u0 + (i+1) du,
 * likewise in v; outside the grid the gain and its derivatives are 0.  Also returns the
 * partial derivatives dG/du, dG/dv of the interpolant inside the cell. */
static void antenna_gain(const or_radar *rd, double u, double v, double g[2], double gu[2],
                         double gv[2]) {
    g[0] = g[1] = gu[0] = gu[1] = gv[0] = gv[1] = 0.0;
    double fu = (u - rd->ant_u0) / rd->ant_du;
    double fv = (v - rd->ant_v0) / rd->ant_dv;
    double iu = floor(fu), iv = floor(fv);
    if (!(iu >= 0.0 && iu <= (double)(rd->ant_nu - 2) && iv >= 0.0 && iv <= (double)(rd->ant_nv - 2)))
        return;
    double tu = fu - iu, tv = fv - iv;
    int64_t i = (int64_t)iu, j = (int64_t)iv;
    const double *g00 = rd->ant + ((size_t)j * rd->ant_nu + i) * 2;
    const double *g10 = g00 + 2;                         /* u + du */
    const double *g01 = g00 + (size_t)rd->ant_nu * 2;    /* v + dv */
    const double *g11 = g01 + 2;
    for (int c = 0; c < 2; ++c) {
        g[c] = (1.0 - tv) * ((1.0 - tu) * g00[c] + tu * g10[c]) + tv * ((1.0 - tu) * g01[c] + tu * g11[c]);
        gu[c] = ((1.0 - tv) * (g10[c] - g00[c]) + tv * (g11[c] - g01[c])) / rd->ant_du;
        gv[c] = ((1.0 - tu) * (g01[c] - g00[c]) + tu * (g11[c] - g10[c])) / rd->ant_dv;
    }
}

int or_version(void) { return 1; }

void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Scatterer n seen from the platform at time t (update_simulation(t) followed by
 * scatterers_range() and scatterers_complex_amplitudes() of Algorithm 1). */
static void echo_at(const or_radar *rd, const or_platform *pf, const or_scene *sc,
                    int64_t n, double t, or_echo *e) {
    double ts = t - sc->t0;
    double sx = sc->origin[0] + (double)sc->x[n] + (double)sc->vx[n] * ts;
    double sy = sc->origin[1] + (double)sc->y[n] + (double)sc->vy[n] * ts;
    double sz = sc->origin[2] + (double)sc->z[n] + (double)sc->vz[n] * ts;
    double px = pf->p0[0] + pf->v[0] * t;
    double py = pf->p0[1] + pf->v[1] * t;
    double pz = pf->p0[2] + pf->v[2] * t;
    double dx = px - sx, dy = py - sy, dz = pz - sz;
    double rho = sqrt(dx * dx + dy * dy);
    double R = sqrt(dx * dx + dy * dy + dz * dz);
    double rref = pf->r_ref0 + pf->r_ref_rate * t;
    /* dR = R - r_ref = (|d|^2 - r_ref^2) / (R + r_ref), with d_z - r_ref taken as
     * (P_z - r_ref) - s_z: the same number as the difference of the two ~8e5 m ranges,
     * without the ~1e-10 m their FP64 rounding leaves in it */
    double dzr = (pz - rref) - sz;
    double dR = (dx * dx + dy * dy + dzr * (dz + rref)) / (R + rref);
    double lambda = rd->c_mps / rd->carrier_hz;
    double theta = atan2(rho, dz);
    double base = sqrt((double)sc->nrcs[n] * sc->area) * (rref / R) * (rref / R);
    double psi = 2.0 * R / lambda;
    double phi = -2.0 * OR_PI * (psi - rint(psi));
    e->R = R;
    e->dR = dR;
    e->rho = rho;
    e->dx = dx;
    e->dy = dy;
    e->dz = dz;
    e->theta = theta;
    e->psi = psi;
    e->base = base;
    e->cr = cos(phi);
    e->ci = sin(phi);
    if (rd->ant_nu > 0) {
        double g[2], gu[2], gv[2];
        e->u = -dx / R;
        e->v = -dy / R;
        antenna_gain(rd, e->u, e->v, g, gu, gv);
        e->g_re = g[0];
        e->g_im = g[1];
        e->gu_re = gu[0];
        e->gu_im = gu[1];
        e->gv_re = gv[0];
        e->gv_im = gv[1];
        e->amp = base * sqrt(g[0] * g[0] + g[1] * g[1]);
        e->re = base * (g[0] * e->cr - g[1] * e->ci);
        e->im = base * (g[0] * e->ci + g[1] * e->cr);
    } else {
        double tb = rd->beamwidth_rad;
        double w = exp(-2.0 * OR_LN2 * theta * theta / (tb * tb));
        e->g_re = w;
        e->g_im = 0.0;
        e->u = e->v = e->gu_re = e->gu_im = e->gv_re = e->gv_im = 0.0;
        e->amp = base * w;
        e->re = e->amp * e->cr;
        e->im = e->amp * e->ci;
    }
}

static double gate_coord_of(const or_radar *rd, double dR) {
    return dR / rd->gate_width_m + 0.5 * (double)rd->n_gates;
}

/* Pulse-pair Doppler of Algorithm 1, D = arg(conj(C2) C1) PRF, as the pre-floor bin
 * coordinate nu N_d + 1/2, nu = -D / (2 pi PRF) in cycles per pulse, in [-1/2, 1/2).
 * With C = |C| G e^{-j 2 pi psi}, psi = 2 R / lambda (G the pattern's complex gain):
 *   arg(conj(C2) C1) = 2 pi (psi2 - psi1) + arg(conj(G2) G1)        (mod 2 pi),
 * so nu = (psi1 - psi2) - arg(conj(G2) G1) / (2 pi), wrapped.  psi1 - psi2 = -2 (R2 - R1) /
 * lambda is taken from the range change over the pair,
 *   R2 - R1 = (|d2|^2 - |d1|^2) / (R1 + R2) = e . (2 d1 + e) / (R1 + R2),
 * e = d2 - d1 = (V - v) / PRF (both ends move linearly over the PRI): the same number as
 * the difference of the two ~7e7-cycle phases, without the ~1e-8 cycles that their FP64
 * rounding leaves in that difference. */
static double bin_coord_of(const or_radar *rd, const or_platform *pf, const or_scene *sc,
                           int64_t n, const or_echo *c1, const or_echo *c2, int n_doppler) {
    double dt = 1.0 / rd->prf_hz;
    double ex = (pf->v[0] - (double)sc->vx[n]) * dt;
    double ey = (pf->v[1] - (double)sc->vy[n]) * dt;
    double ez = (pf->v[2] - (double)sc->vz[n]) * dt;
    double dR21 = (ex * (2.0 * c1->dx + ex) + ey * (2.0 * c1->dy + ey) + ez * (2.0 * c1->dz + ez))
                  / (c1->R + c2->R);
    double lambda = rd->c_mps / rd->carrier_hz;
    double nu = -2.0 * dR21 / lambda;                        /* psi1 - psi2 */
    double gr = c2->g_re * c1->g_re + c2->g_im * c1->g_im;   /* conj(G2) G1 */
    double gi = c2->g_re * c1->g_im - c2->g_im * c1->g_re;
    nu -= atan2(gi, gr) / (2.0 * OR_PI);
    nu -= floor(nu + 0.5);
    return nu * (double)n_doppler + 0.5;
}

static int64_t pmod64(int64_t a, int64_t m) {
    int64_t r = a % m;
    return r < 0 ? r + m : r;
}

static void neu_add(double *s, double *c, double v) {
    double t = *s + v;
    if (fabs(*s) >= fabs(v)) *c += (*s - t) + v;
    else *c += (v - t) + *s;
    *s = t;
}

/* Per-scatterer state at time t for n in [n0, n0+count): used by tests. */
void or_echo_batch(const or_radar *rd, const or_platform *pf, const or_scene *sc, double t,
                   int64_t n0, int64_t count, double *R, double *dR, double *theta,
                   double *amp, double *c_re, double *c_im) {
    for (int64_t j = 0; j < count; ++j) {
        or_echo e;
        echo_at(rd, pf, sc, n0 + j, t, &e);
        if (R) R[j] = e.R;
        if (dR) dR[j] = e.dR;
        if (theta) theta[j] = e.theta;
        if (amp) amp[j] = e.amp;
        if (c_re) c_re[j] = e.re;
        if (c_im) c_im[j] = e.im;
    }
}

/* Gate and Doppler bin of every scatterer for the pulse pair (p, p+1), with the
 * pre-floor coordinates (for index-exactness checks). */
void or_cells(const or_radar *rd, const or_platform *pf, const or_scene *sc, int64_t pulse,
              int32_t n_doppler, int32_t *gate, int32_t *bin, double *gate_coord, double *bin_coord) {
    double t1 = (double)pulse / rd->prf_hz;
    double t2 = (double)(pulse + 1) / rd->prf_hz;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < sc->n; ++n) {
        or_echo e1, e2;
        echo_at(rd, pf, sc, n, t1, &e1);
        echo_at(rd, pf, sc, n, t2, &e2);
        double gc = gate_coord_of(rd, e1.dR);
        double bc = bin_coord_of(rd, pf, sc, n, &e1, &e2, n_doppler);
        if (gate_coord) gate_coord[n] = gc;
        if (bin_coord) bin_coord[n] = bc;
        if (gate) gate[n] = (int32_t)floor(gc);
        if (bin) bin[n] = (int32_t)pmod64((int64_t)floor(bc), n_doppler);
    }
}

/* Regular mode (n_fast = 0): Y[p - pulse0, g] = sum_n C_n(t_p) over scatterers in gate g.
 * iq: [n_pulses][n_gates][2] doubles, overwritten. */
void or_direct_sum(const or_radar *rd, const or_platform *pf, const or_scene *sc,
                   int64_t pulse0, int32_t n_pulses, double *iq) {
    const int G = rd->n_gates;
    const int64_t N = sc->n;
    const int64_t csz = (N + OR_NCHUNK - 1) / OR_NCHUNK;
    double *part = (double *)calloc((size_t)OR_NCHUNK * G * 4, sizeof(double));
    for (int32_t p = 0; p < n_pulses; ++p) {
        double t = (double)(pulse0 + p) / rd->prf_hz;
        memset(part, 0, sizeof(double) * (size_t)OR_NCHUNK * G * 4);
#pragma omp parallel for schedule(static)
        for (int ch = 0; ch < OR_NCHUNK; ++ch) {
            double *pp = part + (size_t)ch * G * 4;
            int64_t lo = ch * csz, hi = lo + csz < N ? lo + csz : N;
            for (int64_t n = lo; n < hi; ++n) {
                or_echo e;
                echo_at(rd, pf, sc, n, t, &e);
                double g = floor(gate_coord_of(rd, e.dR));
                if (g < 0.0 || g >= (double)G) continue;
                int gi = (int)g;
                neu_add(&pp[gi * 4 + 0], &pp[gi * 4 + 1], e.re);
                neu_add(&pp[gi * 4 + 2], &pp[gi * 4 + 3], e.im);
            }
        }
        for (int g = 0; g < G; ++g) {
            double sr = 0, cr = 0, si = 0, ci = 0;
            for (int ch = 0; ch < OR_NCHUNK; ++ch) {
                const double *pp = part + (size_t)ch * G * 4 + g * 4;
                neu_add(&sr, &cr, pp[0]);
                neu_add(&sr, &cr, pp[1]);
                neu_add(&si, &ci, pp[2]);
                neu_add(&si, &ci, pp[3]);
            }
            iq[((size_t)p * G + g) * 2 + 0] = sr + cr;
            iq[((size_t)p * G + g) * 2 + 1] = si + ci;
        }
    }
    free(part);
}

/* Fast mode, Algorithm 1: Doppler spectra of updates update0 .. update0+n_updates-1.
 * T: [n_updates][n_gates][n_doppler][2] doubles, overwritten. */
void or_doppler_spectra(const or_radar *rd, const or_platform *pf, const or_scene *sc,
                        int64_t update0, int32_t n_updates, int32_t n_fast, int32_t n_doppler,
                        double *T) {
    const int G = rd->n_gates;
    const int K = n_doppler;
    const int64_t cells = (int64_t)G * K;
    const int64_t N = sc->n;
    const int64_t csz = (N + OR_NCHUNK - 1) / OR_NCHUNK;
    double *part = (double *)malloc(sizeof(double) * (size_t)OR_NCHUNK * cells * 4);
    for (int32_t u = 0; u < n_updates; ++u) {
        int64_t p_i = (update0 + u) * (int64_t)n_fast;
        double t_i = (double)p_i / rd->prf_hz;            /* update_simulation(i n_fast / PRF) */
        double t_n = (double)(p_i + 1) / rd->prf_hz;      /* update_simulation((i n_fast + 1) / PRF) */
        memset(part, 0, sizeof(double) * (size_t)OR_NCHUNK * cells * 4);
#pragma omp parallel for schedule(static)
        for (int ch = 0; ch < OR_NCHUNK; ++ch) {
            double *pp = part + (size_t)ch * cells * 4;
            int64_t lo = ch * csz, hi = lo + csz < N ? lo + csz : N;
            for (int64_t n = lo; n < hi; ++n) {
                or_echo ci, cn;
                echo_at(rd, pf, sc, n, t_i, &ci);   /* C_i, R_i */
                echo_at(rd, pf, sc, n, t_n, &cn);   /* C_{i+1} */
                double g = floor(gate_coord_of(rd, ci.dR));
                if (g < 0.0 || g >= (double)G) continue;
                int64_t k = pmod64((int64_t)floor(bin_coord_of(rd, pf, sc, n, &ci, &cn, K)), K);
                int64_t cell = (int64_t)g * K + k;   /* rasterize(C_i, T, i, R_i, D_i) */
                neu_add(&pp[cell * 4 + 0], &pp[cell * 4 + 1], ci.re);
                neu_add(&pp[cell * 4 + 2], &pp[cell * 4 + 3], ci.im);
            }
        }
        double *Tu = T + (size_t)u * cells * 2;
#pragma omp parallel for schedule(static)
        for (int64_t cell = 0; cell < cells; ++cell) {
            double sr = 0, cr = 0, si = 0, cci = 0;
            for (int ch = 0; ch < OR_NCHUNK; ++ch) {
                const double *pp = part + (size_t)ch * cells * 4 + cell * 4;
                neu_add(&sr, &cr, pp[0]);
                neu_add(&sr, &cr, pp[1]);
                neu_add(&si, &cci, pp[2]);
                neu_add(&si, &cci, pp[3]);
            }
            Tu[cell * 2 + 0] = sr + cr;
            Tu[cell * 2 + 1] = si + cci;
        }
    }
    free(part);
}

/* Unnormalised 1-D DFT along the last axis of [n_rows][n][2]:
 * out[r, m] = sum_k in[r, k] exp(sign j 2 pi k m / n).  sign = +1: the inverse
 * transform of the post-processing step; sign = -1: its adjoint. */
static void dft_rows(const double *in, int64_t n_rows, int32_t n, int sign, double *out) {
    double *tw = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    for (int r = 0; r < n; ++r) {
        tw[2 * r + 0] = cos(2.0 * OR_PI * (double)r / (double)n);
        tw[2 * r + 1] = sin(2.0 * OR_PI * (double)r / (double)n) * (double)sign;
    }
#pragma omp parallel for schedule(static)
    for (int64_t row = 0; row < n_rows; ++row) {
        const double *a = in + (size_t)row * n * 2;
        double *b = out + (size_t)row * n * 2;
        for (int m = 0; m < n; ++m) {
            double sr = 0, cr = 0, si = 0, ci = 0;
            for (int k = 0; k < n; ++k) {
                int r = (int)(((int64_t)k * m) % n);
                double wr = tw[2 * r], wi = tw[2 * r + 1];
                neu_add(&sr, &cr, a[2 * k] * wr - a[2 * k + 1] * wi);
                neu_add(&si, &ci, a[2 * k] * wi + a[2 * k + 1] * wr);
            }
            b[2 * m + 0] = sr + cr;
            b[2 * m + 1] = si + ci;
        }
    }
    free(tw);
}

void or_ifft(const double *T, int64_t n_rows, int32_t n_doppler, double *s) {
    dft_rows(T, n_rows, n_doppler, +1, s);
}

void or_dft(const double *s, int64_t n_rows, int32_t n_doppler, double *T) {
    dft_rows(s, n_rows, n_doppler, -1, T);
}

/* Blend weight of a spectrum at normalised distance d = |p_i - x| / n_fast.
 * window 0: Eq. (1), (1 - d)^(1/2);  1: cos(pi d / 2) (the squared weights are a
 * raised cosine);  2: 1 - d (linear amplitude, test window).  Zero for d > 1. */
double or_window(int32_t window, double d) {
    if (d < 0.0) d = -d;
    if (d >= 1.0) return 0.0;   /* every window vanishes at the neighbouring update */
    switch (window) {
    case 0: return sqrt(1.0 - d);
    case 1: return cos(0.5 * OR_PI * d);
    case 2: return 1.0 - d;
    default: return NAN;
    }
}

/* Post-processing steps 2-4 of Section III.B for pulses pulse0 .. pulse0+n_pulses-1.
 * T holds spectra of updates update0 .. update0+S-1 ([S][n_gates][n_doppler][2]).
 * iq: [n_pulses][n_gates][2], overwritten.  Returns 0, or -1 when a pulse needs
 * a spectrum with non-zero weight that is not in T. */
int or_synth(int32_t n_gates, const double *T, int32_t S, int64_t update0, int32_t n_fast,
             int32_t n_doppler, int64_t pulse0, int32_t n_pulses, int32_t window, double *iq) {
    const int G = n_gates, K = n_doppler;
    double *s = (double *)malloc(sizeof(double) * (size_t)S * G * K * 2);
    or_ifft(T, (int64_t)S * G, K, s);                       /* step 2: batched iFFT */
    int bad = 0;
    for (int32_t p = 0; p < n_pulses && !bad; ++p) {
        int64_t x = pulse0 + p;
        int64_t i0 = x / n_fast;                            /* floor for x >= 0 */
        for (int g = 0; g < G; ++g) {
            double yr = 0.0, yi = 0.0;
            for (int64_t i = i0 - 1; i <= i0 + 1; ++i) {
                int64_t p_i = i * (int64_t)n_fast;
                double w = or_window(window, (double)(p_i - x) / (double)n_fast);  /* step 3: Eq. (1) */
                if (w == 0.0) continue;
                if (i < update0 || i >= update0 + S) { bad = 1; break; }
                int64_t m = pmod64(x - p_i, K);
                const double *sv = s + (((size_t)(i - update0) * G + g) * K + m) * 2;
                yr += w * sv[0];                            /* step 4: sum into Y */
                yi += w * sv[1];
            }
            iq[((size_t)p * G + g) * 2 + 0] = yr;
            iq[((size_t)p * G + g) * 2 + 1] = yi;
        }
    }
    free(s);
    return bad ? -1 : 0;
}

/* Adjoint of or_synth (PyTorch complex-gradient convention, grad = dL/dRe + j dL/dIm):
 * G_s[i, g, m] = sum_x W_i(x) G_Y[x, g] [ (x - p_i) mod N_d = m ],
 * G_T[i, g, k] = sum_m G_s[i, g, m] exp(-j 2 pi k m / N_d).
 * G_T: [S][n_gates][n_doppler][2], overwritten. */
void or_synth_grad(int32_t n_gates, const double *G_Y, int32_t S, int64_t update0, int32_t n_fast,
                   int32_t n_doppler, int64_t pulse0, int32_t n_pulses, int32_t window, double *G_T) {
    const int G = n_gates, K = n_doppler;
    double *gs = (double *)calloc((size_t)S * G * K * 2, sizeof(double));
    for (int32_t p = 0; p < n_pulses; ++p) {
        int64_t x = pulse0 + p;
        int64_t i0 = x / n_fast;
        for (int64_t i = i0 - 1; i <= i0 + 1; ++i) {
            if (i < update0 || i >= update0 + S) continue;
            int64_t p_i = i * (int64_t)n_fast;
            double w = or_window(window, (double)(p_i - x) / (double)n_fast);
            if (w == 0.0) continue;
            int64_t m = pmod64(x - p_i, K);
            for (int g = 0; g < G; ++g) {
                double *d = gs + (((size_t)(i - update0) * G + g) * K + m) * 2;
                d[0] += w * G_Y[((size_t)p * G + g) * 2 + 0];
                d[1] += w * G_Y[((size_t)p * G + g) * 2 + 1];
            }
        }
    }
    or_dft(gs, (int64_t)S * G, K, G_T);
    free(gs);
}

/* dC/dz of scatterer echo e (C = a exp(j phi)): C (dln a/dz + j dphi/dz) with
 * dR/dz = -d_z / R, dtheta/dz = rho / R^2.  With the tabulated pattern, C = base G e^{j phi}
 * and the pattern term is base e^{j phi} (dG/du du/dz + dG/dv dv/dz), where
 * u = -d_x / R gives du/dz = u d_z / R^2 (likewise v). */
static void dC_dz(const or_radar *rd, const or_echo *e, double *dre, double *dim) {
    double lambda = rd->c_mps / rd->carrier_hz;
    double R2 = e->R * e->R;
    double dphi = 4.0 * OR_PI * e->dz / (lambda * e->R);
    if (rd->ant_nu > 0) {
        double dlna = 2.0 * e->dz / R2;   /* (r_ref / R)^2 factor only */
        *dre = e->re * dlna - e->im * dphi;
        *dim = e->im * dlna + e->re * dphi;
        double du = e->u * e->dz / R2, dv = e->v * e->dz / R2;
        double dg_re = e->gu_re * du + e->gv_re * dv;
        double dg_im = e->gu_im * du + e->gv_im * dv;
        *dre += e->base * (dg_re * e->cr - dg_im * e->ci);
        *dim += e->base * (dg_re * e->ci + dg_im * e->cr);
        return;
    }
    double tb = rd->beamwidth_rad;
    double dlna = -4.0 * OR_LN2 * e->theta / (tb * tb) * (e->rho / R2) + 2.0 * e->dz / R2;
    *dre = e->re * dlna - e->im * dphi;
    *dim = e->im * dlna + e->re * dphi;
}

/* The tabulated pattern and its partial derivatives at (u, v) (for the tests). */
void or_antenna_gain(const or_radar *rd, double u, double v, double *g, double *gu, double *gv) {
    antenna_gain(rd, u, v, g, gu, gv);
}

/* Adjoint of the fast-mode rasterisation: for each scatterer, the gradient of a
 * real loss w.r.t. its height z and NRCS given G_T = dL/dT ([n_updates][G][K][2]).
 * grad_z, grad_nrcs: [n] doubles, overwritten.  Index functions (gate, bin) are
 * piecewise constant and contribute no gradient. */
void or_fast_grad(const or_radar *rd, const or_platform *pf, const or_scene *sc,
                  int64_t update0, int32_t n_updates, int32_t n_fast, int32_t n_doppler,
                  const double *G_T, double *grad_z, double *grad_nrcs) {
    const int G = rd->n_gates, K = n_doppler;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < sc->n; ++n) {
        double gz = 0.0, gsig = 0.0;
        for (int32_t u = 0; u < n_updates; ++u) {
            int64_t p_i = (update0 + u) * (int64_t)n_fast;
            or_echo ci, cn;
            echo_at(rd, pf, sc, n, (double)p_i / rd->prf_hz, &ci);
            echo_at(rd, pf, sc, n, (double)(p_i + 1) / rd->prf_hz, &cn);
            double g = floor(gate_coord_of(rd, ci.dR));
            if (g < 0.0 || g >= (double)G) continue;
            int64_t k = pmod64((int64_t)floor(bin_coord_of(rd, pf, sc, n, &ci, &cn, K)), K);
            const double *gt = G_T + (((size_t)u * G + (int64_t)g) * K + k) * 2;
            double dre, dim;
            dC_dz(rd, &ci, &dre, &dim);
            gz += gt[0] * dre + gt[1] * dim;                 /* Re(conj(G) dC/dz) */
            double sig = (double)sc->nrcs[n];
            if (sig > 0.0) gsig += (gt[0] * ci.re + gt[1] * ci.im) / (2.0 * sig);
        }
        grad_z[n] = gz;
        grad_nrcs[n] = gsig;
    }
}

/* Adjoint of the regular-mode summation given G_Y = dL/dY ([n_pulses][G][2]). */
void or_direct_grad(const or_radar *rd, const or_platform *pf, const or_scene *sc,
                    int64_t pulse0, int32_t n_pulses, const double *G_Y,
                    double *grad_z, double *grad_nrcs) {
    const int G = rd->n_gates;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < sc->n; ++n) {
        double gz = 0.0, gsig = 0.0;
        for (int32_t p = 0; p < n_pulses; ++p) {
            or_echo e;
            echo_at(rd, pf, sc, n, (double)(pulse0 + p) / rd->prf_hz, &e);
            double g = floor(gate_coord_of(rd, e.dR));
            if (g < 0.0 || g >= (double)G) continue;
            const double *gy = G_Y + ((size_t)p * G + (int64_t)g) * 2;
            double dre, dim;
            dC_dz(rd, &e, &dre, &dim);
            gz += gy[0] * dre + gy[1] * dim;
            double sig = (double)sc->nrcs[n];
            if (sig > 0.0) gsig += (gy[0] * e.re + gy[1] * e.im) / (2.0 * sig);
        }
        grad_z[n] = gz;
        grad_nrcs[n] = gsig;
    }
}

/* Regular mode with the gate decisions supplied (gate[p * n + j] for pulse pulse0 + p,
 * scatterer j): sums the FP64 amplitudes C_j(t_p) into those gates.  Lets a test compare
 * sums with an implementation whose gate decisions were taken in another precision
 * (a decision whose coordinate is within rounding of a gate edge may go either way). */
void or_direct_sum_cells(const or_radar *rd, const or_platform *pf, const or_scene *sc,
                         int64_t pulse0, int32_t n_pulses, const int32_t *gate, double *iq) {
    const int G = rd->n_gates;
    const int64_t N = sc->n;
    const int64_t csz = (N + OR_NCHUNK - 1) / OR_NCHUNK;
    double *part = (double *)calloc((size_t)OR_NCHUNK * G * 4, sizeof(double));
    for (int32_t p = 0; p < n_pulses; ++p) {
        double t = (double)(pulse0 + p) / rd->prf_hz;
        const int32_t *gp = gate + (size_t)p * N;
        memset(part, 0, sizeof(double) * (size_t)OR_NCHUNK * G * 4);
#pragma omp parallel for schedule(static)
        for (int ch = 0; ch < OR_NCHUNK; ++ch) {
            double *pp = part + (size_t)ch * G * 4;
            int64_t lo = ch * csz, hi = lo + csz < N ? lo + csz : N;
            for (int64_t n = lo; n < hi; ++n) {
                int gi = gp[n];
                if (gi < 0 || gi >= G) continue;
                or_echo e;
                echo_at(rd, pf, sc, n, t, &e);
                neu_add(&pp[gi * 4 + 0], &pp[gi * 4 + 1], e.re);
                neu_add(&pp[gi * 4 + 2], &pp[gi * 4 + 3], e.im);
            }
        }
        for (int g = 0; g < G; ++g) {
            double sr = 0, cr = 0, si = 0, ci = 0;
            for (int ch = 0; ch < OR_NCHUNK; ++ch) {
                const double *pp = part + (size_t)ch * G * 4 + g * 4;
                neu_add(&sr, &cr, pp[0]);
                neu_add(&sr, &cr, pp[1]);
                neu_add(&si, &ci, pp[2]);
                neu_add(&si, &ci, pp[3]);
            }
            iq[((size_t)p * G + g) * 2 + 0] = sr + cr;
            iq[((size_t)p * G + g) * 2 + 1] = si + ci;
        }
    }
    free(part);
}

/* Fast-mode rasterisation of Algorithm 1 with the (gate, bin) decisions supplied
 * (gate[u * n + j], bin[u * n + j] for update update0 + u): T[u, gate, bin] += C_j(t_{p_u}). */
void or_doppler_spectra_cells(const or_radar *rd, const or_platform *pf, const or_scene *sc,
                              int64_t update0, int32_t n_updates, int32_t n_fast,
                              int32_t n_doppler, const int32_t *gate, const int32_t *bin,
                              double *T) {
    const int G = rd->n_gates;
    const int K = n_doppler;
    const int64_t cells = (int64_t)G * K;
    const int64_t N = sc->n;
    const int64_t csz = (N + OR_NCHUNK - 1) / OR_NCHUNK;
    double *part = (double *)malloc(sizeof(double) * (size_t)OR_NCHUNK * cells * 4);
    for (int32_t u = 0; u < n_updates; ++u) {
        int64_t p_i = (update0 + u) * (int64_t)n_fast;
        double t_i = (double)p_i / rd->prf_hz;
        const int32_t *gu = gate + (size_t)u * N;
        const int32_t *bu = bin + (size_t)u * N;
        memset(part, 0, sizeof(double) * (size_t)OR_NCHUNK * cells * 4);
#pragma omp parallel for schedule(static)
        for (int ch = 0; ch < OR_NCHUNK; ++ch) {
            double *pp = part + (size_t)ch * cells * 4;
            int64_t lo = ch * csz, hi = lo + csz < N ? lo + csz : N;
            for (int64_t n = lo; n < hi; ++n) {
                int32_t g = gu[n], k = bu[n];
                if (g < 0 || g >= G || k < 0 || k >= K) continue;
                or_echo ci;
                echo_at(rd, pf, sc, n, t_i, &ci);
                int64_t cell = (int64_t)g * K + k;
                neu_add(&pp[cell * 4 + 0], &pp[cell * 4 + 1], ci.re);
                neu_add(&pp[cell * 4 + 2], &pp[cell * 4 + 3], ci.im);
            }
        }
        double *Tu = T + (size_t)u * cells * 2;
#pragma omp parallel for schedule(static)
        for (int64_t cell = 0; cell < cells; ++cell) {
            double sr = 0, cr = 0, si = 0, cci = 0;
            for (int ch = 0; ch < OR_NCHUNK; ++ch) {
                const double *pp = part + (size_t)ch * cells * 4 + cell * 4;
                neu_add(&sr, &cr, pp[0]);
                neu_add(&sr, &cr, pp[1]);
                neu_add(&si, &cci, pp[2]);
                neu_add(&si, &cci, pp[3]);
            }
            Tu[cell * 2 + 0] = sr + cr;
            Tu[cell * 2 + 1] = si + cci;
        }
    }
    free(part);
}
