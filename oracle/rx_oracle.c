/*
 * FP64 CPU oracle of the receiver DSP chain -- TEST INFRASTRUCTURE ONLY.
 *
 * Used by the tests, the smoke check and the benchmark's CPU-baseline leg; the
 * CUDA receiver never links or calls it and shares no code with it.  Plain
 * loops in the order of the method, double precision throughout.
 *
 * Paper passages followed (Sec. 2, "Multi-Format Real-Time DSP in GPU"):
 *  - 12-bit ADC buffers of 2^22 samples at 4 GS/s, processed buffer by buffer
 *    with overlap-save continuity carried from the previous buffer;
 *  - KK front end: square root and natural logarithm of the detected signal at
 *    4 samples/symbol, FD Hilbert transform by FFT/IFFT to recover the phase,
 *    mixing with the square-root term and frequency downshifting (Fig. 1d);
 *  - filtering and reduction to 2 samples/symbol, then a decision-directed LMS
 *    equaliser with symbol-phase recovery, decision and demapping, applied to
 *    data blocks of each buffer in parallel;
 *  - PAM: equalisation, symbol decision and demapping (Fig. 1b);
 *  - performance as Q-factor derived from the BER (Sec. 3).
 * The filter shapes, adaptive algorithms (CMA, LMS, blind phase search) and
 * their parameters are the configured workload's; where the paper is silent the
 * reading used is stated beside the code.
 */
#include "rx_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

typedef struct { double re, im; } cx;

static cx cx_mk(double r, double i) { cx z; z.re = r; z.im = i; return z; }
static cx cx_add(cx a, cx b) { return cx_mk(a.re + b.re, a.im + b.im); }
static cx cx_sub(cx a, cx b) { return cx_mk(a.re - b.re, a.im - b.im); }
static cx cx_mul(cx a, cx b) { return cx_mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
static cx cx_conj(cx a) { return cx_mk(a.re, -a.im); }
static cx cx_scale(cx a, double s) { return cx_mk(a.re * s, a.im * s); }
static double cx_abs2(cx a) { return a.re * a.re + a.im * a.im; }
static cx cx_expj(double t) { return cx_mk(cos(t), sin(t)); }

static void *xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

/* ------------------------------------------------------------- 12-bit unpack
 * Two 12-bit samples per three bytes (the ADC word of Sec. 2).  order 0:
 * little-endian 24-bit word; order 1: big-endian nibble order. */
void orx_unpack(const uint8_t *in, int64_t nsamp, int order, int32_t *codes)
{
    for (int64_t p = 0; p < nsamp / 2; p++) {
        uint32_t b0 = in[3 * p], b1 = in[3 * p + 1], b2 = in[3 * p + 2];
        if (order == 0) {
            codes[2 * p] = (int32_t)(b0 | ((b1 & 0x0Fu) << 8));
            codes[2 * p + 1] = (int32_t)((b1 >> 4) | (b2 << 4));
        } else {
            codes[2 * p] = (int32_t)((b0 << 4) | (b1 >> 4));
            codes[2 * p + 1] = (int32_t)(((b1 & 0x0Fu) << 8) | b2);
        }
    }
}

/* ------------------------------------------------------------------- FFT
 * Radix-2 decimation-in-time, in place.  forward: X_k = sum x_n e^{-2pi i nk/N};
 * inverse: x_n = (1/N) sum X_k e^{+2pi i nk/N}.  Twiddles from cos/sin of the
 * exact angle (no recurrence). */
void orx_fft(double *re, double *im, int n, int inverse)
{
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    double sgn = inverse ? 1.0 : -1.0;
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1;
        for (int k = 0; k < half; k++) {
            double ang = sgn * 2.0 * PI * (double)k / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int s = 0; s < n; s += len) {
                int a = s + k, b = a + half;
                double xr = re[b] * wr - im[b] * wi;
                double xi = re[b] * wi + im[b] * wr;
                re[b] = re[a] - xr; im[b] = im[a] - xi;
                re[a] += xr; im[a] += xi;
            }
        }
    }
    if (inverse) {
        double s = 1.0 / (double)n;
        for (int i = 0; i < n; i++) { re[i] *= s; im[i] *= s; }
    }
}

/* Hilbert transform of one real block, circular: phi = IFFT(FFT(u) * h) with
 * h_k = -j (0 < k < N/2), +j (N/2 < k < N), 0 at k = 0 and k = N/2.
 * (FD Hilbert transform by FFT and IFFT, Sec. 2 KK chain.) */
static void hilbert_block(const double *u, double *phi, int n, double *re, double *im)
{
    for (int i = 0; i < n; i++) { re[i] = u[i]; im[i] = 0.0; }
    orx_fft(re, im, n, 0);
    for (int k = 0; k < n; k++) {
        double a = re[k], b = im[k];
        if (k == 0 || 2 * k == n) { re[k] = 0.0; im[k] = 0.0; }
        else if (2 * k < n) { re[k] = b; im[k] = -a; }      /* times -j */
        else { re[k] = -b; im[k] = a; }                      /* times +j */
    }
    orx_fft(re, im, n, 1);
    for (int i = 0; i < n; i++) phi[i] = re[i];
}

void orx_hilbert_circ(const double *u, double *phi, int n)
{
    double *re = xcalloc((size_t)n, sizeof(double)), *im = xcalloc((size_t)n, sizeof(double));
    hilbert_block(u, phi, n, re, im);
    free(re); free(im);
}

/* Intensity -> KK field, log guard as in the receiver. */
static double kk_intensity(int32_t code) { return code > 0 ? (double)code : 0.5; }

/* One circular KK reconstruction: E = sqrt(I) exp(j H{ln(I)/2}). */
void orx_kk_circ(const double *intensity, double *e_re, double *e_im, int n)
{
    double *u = xcalloc((size_t)n, sizeof(double)), *phi = xcalloc((size_t)n, sizeof(double));
    for (int i = 0; i < n; i++) u[i] = 0.5 * log(intensity[i]);
    orx_hilbert_circ(u, phi, n);
    for (int i = 0; i < n; i++) {
        double a = sqrt(intensity[i]);
        e_re[i] = a * cos(phi[i]);
        e_im[i] = a * sin(phi[i]);
    }
    free(u); free(phi);
}

/* Root-raised cosine, sps*span+1 taps, unit energy, zero phase. */
void orx_rrc(double beta, int sps, int span, double *taps) { orx_rrc_half(beta, sps, sps * span / 2, taps); }

/* The same pulse with 2*half+1 taps (any half-length). */
void orx_rrc_half(double beta, int sps, int half, double *taps)
{
    int n = 2 * half + 1;
    double e = 0.0;
    for (int i = 0; i < n; i++) {
        double t = (double)(i - half) / (double)sps, v;
        if (fabs(t) < 1e-12)
            v = 1.0 - beta + 4.0 * beta / PI;
        else if (beta > 0.0 && fabs(fabs(4.0 * beta * t) - 1.0) < 1e-12)
            v = beta / sqrt(2.0) * ((1.0 + 2.0 / PI) * sin(PI / (4.0 * beta)) +
                                    (1.0 - 2.0 / PI) * cos(PI / (4.0 * beta)));
        else
            v = (sin(PI * t * (1.0 - beta)) + 4.0 * beta * t * cos(PI * t * (1.0 + beta))) /
                (PI * t * (1.0 - 16.0 * beta * beta * t * t));
        taps[i] = v;
        e += v * v;
    }
    e = 1.0 / sqrt(e);
    for (int i = 0; i < n; i++) taps[i] *= e;
}

/* ------------------------------------------- frequency-domain filtering
 * The paper's static equaliser runs in the frequency domain on overlap-save
 * blocks of a 1024-point FFT, and a 512-point IFFT brings the signal to 2
 * samples per symbol (Sec. 2, KK chain).  Readings: "100% overlap" is a hop of
 * N/2 (8192 blocks per 2^22-sample buffer); the filter is zero-phase and its
 * response is H_k = sum_i h_i e^{-2 pi i k i / N} over the taps i = -(L-1)/2 ..
 * (L-1)/2; the downsampler keeps the bins -N/4 <= k < N/4 (bin k goes to
 * position k mod N/2 of the half-length spectrum); block b takes the N inputs
 * starting at stream index hop*b - N/4 and keeps its central half. */
void orx_fd_response(const double *h, int ntaps, int n, double *H_re, double *H_im)
{
    int half = (ntaps - 1) / 2;
    for (int k = 0; k < n; k++) {
        double re = 0.0, im = 0.0;
        for (int i = -half; i <= half; i++) {
            double a = -2.0 * PI * (double)(((int64_t)k * i) % n) / (double)n;
            re += h[i + half] * cos(a);
            im += h[i + half] * sin(a);
        }
        H_re[k] = re;
        H_im[k] = im;
    }
}

/* One block: X = FFT_N(x); Z_{k mod N/2} = X_k H_k for -N/4 <= k < N/4;
 * z_m = (1/N) sum_k' Z_k' e^{+2 pi i k' m / (N/2)}, which for a block with no
 * energy outside those bins is the circular convolution of x with h at the even
 * index 2m; y = z_m for m in [N/8, 3N/8) (N/4 outputs). */
void orx_fd_block(const double *x_re, const double *x_im, int n, const double *H_re, const double *H_im,
                  double *y_re, double *y_im)
{
    int m2 = n / 2;
    double *re = xcalloc((size_t)n, sizeof(double)), *im = xcalloc((size_t)n, sizeof(double));
    double *zr = xcalloc((size_t)m2, sizeof(double)), *zi = xcalloc((size_t)m2, sizeof(double));
    for (int i = 0; i < n; i++) { re[i] = x_re[i]; im[i] = x_im[i]; }
    orx_fft(re, im, n, 0);
    for (int kp = 0; kp < m2; kp++) {
        int k = kp < n / 4 ? kp : kp + m2;
        zr[kp] = re[k] * H_re[k] - im[k] * H_im[k];
        zi[kp] = re[k] * H_im[k] + im[k] * H_re[k];
    }
    orx_fft(zr, zi, m2, 1);          /* includes 1/(N/2) */
    for (int m = n / 8; m < 3 * n / 8; m++) {
        y_re[m - n / 8] = 0.5 * zr[m];
        y_im[m - n / 8] = 0.5 * zi[m];
    }
    free(re); free(im); free(zr); free(zi);
}

/* The same block without downsampling (the PAM chain, already at 2 samples per
 * symbol): y = IFFT_N(X H) at the central indices N/4 .. 3N/4 - 1 (N/2 outputs),
 * the circular convolution of x with h there, alias-free while the taps span at
 * most N/2 + 1. */
void orx_fd_block_full(const double *x_re, const double *x_im, int n, const double *H_re, const double *H_im,
                       double *y_re, double *y_im)
{
    double *re = xcalloc((size_t)n, sizeof(double)), *im = xcalloc((size_t)n, sizeof(double));
    for (int i = 0; i < n; i++) { re[i] = x_re[i]; im[i] = x_im[i]; }
    orx_fft(re, im, n, 0);
    for (int k = 0; k < n; k++) {
        double a = re[k] * H_re[k] - im[k] * H_im[k], b = re[k] * H_im[k] + im[k] * H_re[k];
        re[k] = a; im[k] = b;
    }
    orx_fft(re, im, n, 1);           /* includes 1/N */
    for (int m = n / 4; m < 3 * n / 4; m++) { y_re[m - n / 4] = re[m]; y_im[m - n / 4] = im[m]; }
    free(re); free(im);
}

/* ----------------------------------------------------------- resampler
 * The paper's ADC is clocked independently of the transmitter; its DSP recovers
 * the clock phase block by block (Sec. 2).  Here the clock relation is a
 * configured integer accumulator (reading): nominal sample m of the transmitter's
 * grid lies at ADC position (rs_phase0 + m rs_step) / 2^32, and the field there is
 * interpolated from the 16 ADC samples around it with a Hann-windowed sinc,
 *   c_j(mu) = sinc(j - mu) (1 + cos(pi (j - mu) / 8)) / 2,  j = -7 .. 8,
 * at the fraction mu rounded down to 10 bits. */
void orx_rs_taps(double mu, double *c)
{
    for (int j = -7; j <= 8; j++) {
        double x = (double)j - mu;
        double sn = fabs(x) < 1e-15 ? 1.0 : sin(PI * x) / (PI * x);
        double w = fabs(x) < 8.0 ? 0.5 * (1.0 + cos(PI * x / 8.0)) : 0.0;
        c[j + 7] = sn * w;
    }
}

/* ---------------------------------------------------- FD clock estimate
 * The paper recovers the clock in the frequency domain block by block and unwraps
 * the clock phase across blocks and buffers (Sec. 2), in the PAM chain after its
 * static FD filter and in the KK chain.  Reading (Godard's band-edge estimator on
 * the FD form's N-point blocks at sps samples/symbol, 4 for KK, 2 for PAM): with
 * Y = FFT(x_b) H / N and S = N / sps the bin of the symbol rate,
 *   C_b = sum_{|k - S/2| <= w} Y_k conj(Y_{k - S}),
 * the correlation of the spectrum at +1/(2T) with its image one symbol rate lower;
 * a symbol grid at ADC positions congruent to d (mod sps) gives
 * arg C_b = -2 pi d / sps.  w is the roll-off half-width ceil(beta S / 2) in bins. */
void orx_fd_clock(const double *x_re, const double *x_im, int n, const double *H_re, const double *H_im,
                  int sps, int w, double *c_re, double *c_im)
{
    double *re = xcalloc((size_t)n, sizeof(double)), *im = xcalloc((size_t)n, sizeof(double));
    for (int i = 0; i < n; i++) { re[i] = x_re[i]; im[i] = x_im[i]; }
    orx_fft(re, im, n, 0);
    double sr = 0.0, si = 0.0;
    const int S = n / sps;
    for (int k = S / 2 - w; k <= S / 2 + w; k++) {
        int kk = ((k % n) + n) % n, km = (((k - S) % n) + n) % n;
        double ar = (re[kk] * H_re[kk] - im[kk] * H_im[kk]) / n, ai = (re[kk] * H_im[kk] + im[kk] * H_re[kk]) / n;
        double br = (re[km] * H_re[km] - im[km] * H_im[km]) / n, bi = (re[km] * H_im[km] + im[km] * H_re[km]) / n;
        sr += ar * br + ai * bi;   /* a conj(b) */
        si += ai * br - ar * bi;
    }
    *c_re = sr; *c_im = si;
    free(re); free(im);
}

/* Clock offset and delay from the block correlations: d_b = -(sps / 2 pi) arg C_b,
 * unwrapped across the blocks (period sps ADC samples, one symbol), then the
 * least-squares line d_b = -tau0 - eps c_b over the block centres c_b (ADC samples):
 * ppm = 1e6 eps, delay = tau0 (in (-sps/2, sps/2], the symbol ambiguity is not
 * resolved). */
int orx_clock_fit(const double *c_re, const double *c_im, const int64_t *center, int nblk, int sps,
                  double *ppm, double *delay)
{
    if (nblk < 2 || sps < 2) return -1;
    const double P = (double)sps, H = 0.5 * P;
    double prev = 0.0, off = 0.0, sx = 0, sy = 0, sxx = 0, sxy = 0;
    double x0 = (double)center[0];
    for (int b = 0; b < nblk; b++) {
        double d = -P / (2.0 * PI) * atan2(c_im[b], c_re[b]);   /* (-sps/2, sps/2] */
        if (b > 0) {
            while (d + off - prev > H) off -= P;
            while (d + off - prev < -H) off += P;
        }
        double y = d + off, x = (double)center[b] - x0;
        prev = y;
        sx += x; sy += y; sxx += x * x; sxy += x * y;
    }
    double nb = (double)nblk, slope = (nb * sxy - sx * sy) / (nb * sxx - sx * sx);
    double icpt = (sy - slope * sx) / nb - slope * x0;   /* at stream index 0 */
    double tau0 = -icpt;
    while (tau0 > H) tau0 -= P;
    while (tau0 <= -H) tau0 += P;
    *ppm = -slope * 1e6;
    *delay = tau0;
    return 0;
}

/* PRBS-15, Fibonacci LFSR x^15 + x^14 + 1; register loaded with
 * (seed mod 32767) + 1; each step outputs r14 xor r15 and shifts it in. */
void orx_prbs15(uint32_t seed, int64_t nbits, uint8_t *out)
{
    uint32_t r = (seed % 32767u) + 1u;
    for (int64_t i = 0; i < nbits; i++) {
        uint32_t nb = ((r >> 13) ^ (r >> 14)) & 1u;
        r = ((r << 1) | nb) & 0x7FFFu;
        out[i] = (uint8_t)nb;
    }
}

/* Q = 20 log10(sqrt(2) erfcinv(2 BER)); erfcinv by bisection on erfc. */
double orx_q_db(double ber)
{
    if (!(ber > 0.0)) return INFINITY;
    if (ber >= 0.5) return -INFINITY;
    double target = 2.0 * ber, lo = 0.0, hi = 30.0;
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (erfc(mid) > target) lo = mid; else hi = mid;
    }
    return 20.0 * log10(sqrt(2.0) * 0.5 * (lo + hi));
}

/* ============================================================ the receiver */
struct orx {
    orx_cfg c;
    int kk, bps, mq, dims, dec, hmf, th;
    double scale, r2;
    double *rrc;
    uint8_t *prbs;                 /* one PRBS-15 period */
    int64_t calls, e_prev, f_prev, q_prev;
    int32_t *chist; int64_t chist_len, chist_cap;
    int have_first; int32_t first_code;
    int flushed;                   /* the stream has ended (orx_flush) */
    int dq_have, dq_prev;          /* differential coding: quadrant of the last decided symbol */
    /* resampler accumulator, piecewise: nominal sample m >= rs_r0 lies at ADC position
     * (rs_psi0 + (m - rs_r0) rs_step) / 2^32; a step change keeps the position of the
     * next nominal sample (orx_set_rs_step) */
    int64_t rs_r0, rs_step;
    __int128 rs_psi0;
    /* clock tracker across calls (clk_track, frequency-domain form): unwrap carry and
     * least-squares sums of the unwrapped block delays since the last reset */
    int ck_have; double ck_y, ck_off, ck_x0;
    int64_t ck_n; double ck_sx, ck_sy, ck_sxx, ck_sxy;
    int64_t pad_calls;             /* pad buffers run by orx_flush (not counted as input) */
    double last_mu, last_sd;       /* PAM: normalisation of the last real buffer */
    cx *ehist; int64_t ehist_start, ehist_len;
    cx *yhist; int64_t yhist_start, yhist_len;
    cx carrier; double gain;
    cx *w;                         /* taps every block of the next call starts from */
    int rs;                        /* resampler to the transmitter's grid */
    int64_t r_prev;                /* nominal field samples emitted */
    cx *rhist; int64_t rhist_start, rhist_len;
    cx *d_R; int64_t d_R_start, d_R_len;
    cx *d_C; int64_t d_C_start, d_C_len;   /* FD clock correlation per emitted block */
    int fd;                        /* frequency-domain reduction to 2 samples/symbol */
    double *fd_Hr, *fd_Hi;         /* its filter response, fd_n bins */
    int trained;
    int have_b, b_last; int64_t m_last;
    int amb_done, amb_r;
    int64_t n_samples, n_symbols, n_bits, n_bit_err, n_sym_err, n_near, n_amb, n_win, n_raw_err, n_slip;
    /* debug views of the last call */
    cx *d_E; int64_t d_E_start, d_E_len;
    cx *d_y; int64_t d_y_start, d_y_len;
    cx *d_z, *d_v; int32_t *d_ahat, *d_draw, *d_berr, *d_near; int64_t d_s_start, d_s_len;
    double *d_win; int64_t d_win_len;
    double scal[5];
};

orx *orx_create(const orx_cfg *cfg)
{
    orx *h = xcalloc(1, sizeof(orx));
    h->c = *cfg;
    int f = cfg->format;
    if (f < 0 || f > 4 || cfg->ntaps < 1 || (!(cfg->ntaps & 1) && cfg->eq_mode != 1) || cfg->win < 1 || cfg->win > 4096 ||
        cfg->eq_mode < 0 || cfg->eq_mode > 1 ||
        (cfg->eq_mode == 1 && (f < 3 || cfg->eq_frozen || cfg->ntaps < 2 || cfg->ntaps > 31)) ||
        cfg->eq_block < cfg->win || cfg->eq_block % cfg->win || cfg->ntrain < 0 || cfg->ntrain % cfg->win ||
        cfg->buf_len < 2 || (cfg->buf_len & 1) || cfg->sps < 2 || (cfg->sps & 1) || cfg->mf_span < 0 ||
        (f >= 3 && (cfg->ncma < 0 || cfg->ncma > cfg->ntrain || cfg->ncma % cfg->win || cfg->bps_b < 1 ||
                    cfg->ds_den < 1 || cfg->ols_n < 4 || (cfg->ols_n & (cfg->ols_n - 1)) ||
                    cfg->ols_v < 2 || (cfg->ols_v & 1) || cfg->ols_v >= cfg->ols_n)) ||
        cfg->mf_mode < 0 || cfg->mf_mode > 1 || cfg->clk_track < 0 || cfg->clk_track > 1 || (cfg->clk_track && cfg->mf_mode != 1) ||
        cfg->diff_code < 0 || cfg->diff_code > 1 || (cfg->diff_code && f < 3) ||
        (cfg->rs_step != 0 && ((f < 3 && cfg->mf_mode == 1) || cfg->rs_step < (int64_t)4252017623LL ||
                               cfg->rs_step > (int64_t)4337916969LL)) ||
        (cfg->mf_mode == 1 && (cfg->sps != (f >= 3 ? 4 : 2) || cfg->fd_n < 16 || (cfg->fd_n & (cfg->fd_n - 1)) ||
                               cfg->fd_taps < 1 || !(cfg->fd_taps & 1) || cfg->fd_taps > cfg->fd_n / 2 + 1))) {
        free(h);
        return NULL;
    }
    h->kk = f >= 3;
    h->bps = (f == 0) ? 1 : (f == 1) ? 2 : (f == 2) ? 3 : (f == 3) ? 2 : 4;
    if (h->kk) {
        h->dims = 2;
        h->mq = (f == 3) ? 2 : 4;
        h->scale = (f == 3) ? sqrt(2.0) : sqrt(10.0);
        h->r2 = (f == 3) ? 1.0 : 1.32;   /* E|a|^4 / E|a|^2 of the unit-power constellation */
        h->dec = cfg->sps / 2;           /* matched filter output at 2 samples/symbol */
    } else {
        h->dims = 1;
        h->mq = 1 << h->bps;
        h->scale = 1.0;
        h->r2 = 0.0;
        h->dec = cfg->sps / 2;
    }
    h->hmf = cfg->sps * cfg->mf_span / 2;
    h->th = (cfg->ntaps - 1) / 2;
    h->rrc = xcalloc((size_t)(2 * h->hmf + 1), sizeof(double));
    orx_rrc(cfg->rrc_beta, cfg->sps, cfg->mf_span, h->rrc);
    h->rs = cfg->rs_step != 0;
    h->rs_r0 = 0;
    h->rs_step = cfg->rs_step;
    h->rs_psi0 = (__int128)cfg->rs_phase0;
    h->fd = cfg->mf_mode == 1;
    if (h->fd) {
        double *hf = xcalloc((size_t)cfg->fd_taps, sizeof(double));
        orx_rrc_half(cfg->rrc_beta, cfg->sps, (cfg->fd_taps - 1) / 2, hf);
        h->fd_Hr = xcalloc((size_t)cfg->fd_n, sizeof(double));
        h->fd_Hi = xcalloc((size_t)cfg->fd_n, sizeof(double));
        orx_fd_response(hf, cfg->fd_taps, cfg->fd_n, h->fd_Hr, h->fd_Hi);
        free(hf);
    }
    h->prbs = xcalloc(32767, 1);
    orx_prbs15(cfg->prbs_seed, 32767, h->prbs);
    h->chist_cap = h->kk ? cfg->ols_n : 2 * h->hmf;
    if (!h->kk && cfg->rs_step != 0 && h->chist_cap < 64) h->chist_cap = 64;   /* the resampler's reach */
    if (!h->kk && cfg->mf_mode == 1 && h->chist_cap < cfg->fd_n) h->chist_cap = cfg->fd_n;
    h->chist = xcalloc((size_t)h->chist_cap, sizeof(int32_t));
    h->w = xcalloc((size_t)cfg->ntaps, sizeof(cx));
    h->w[h->th] = cx_mk(1.0, 0.0);      /* centre tap 1 */
    h->gain = 1.0;
    h->amb_r = -1;
    return h;
}

void orx_set_taps(orx *h, const double *re, const double *im, int n)
{
    for (int i = 0; i < n && i < h->c.ntaps; i++) h->w[i] = cx_mk(re[i], im ? im[i] : 0.0);
}

/* Static frequency-domain filter with given zero-phase taps h_i = re + j im at
 * index i + L, i = -L .. L (Sec. 2: the static FD equalisers' taps come from the
 * link): its N-bin response H_k = sum_i h_i e^{-2 pi i k i / N} replaces the RRC
 * response.  PAM takes the filter output as real, so its taps must be real.
 * Returns 0, or -1 (no FD form, n even or above N/2 + 1, complex PAM taps). */
int orx_set_fd_taps(orx *h, const double *re, const double *im, int n)
{
    if (!h->fd || n < 1 || !(n & 1) || n > h->c.fd_n / 2 + 1) return -1;
    if (!h->kk && im)
        for (int i = 0; i < n; i++)
            if (im[i] != 0.0) return -1;
    int N = h->c.fd_n, half = (n - 1) / 2;
    for (int k = 0; k < N; k++) {
        double hr = 0.0, hi = 0.0;
        for (int i = -half; i <= half; i++) {
            double a = -2.0 * PI * (double)(((int64_t)k * i) % N) / (double)N;
            cx t = cx_mul(cx_mk(re[i + half], im ? im[i + half] : 0.0), cx_expj(a));
            hr += t.re;
            hi += t.im;
        }
        h->fd_Hr[k] = hr;
        h->fd_Hi[k] = hi;
    }
    return 0;
}

/* --------------------------------------------------------------- decisions */
/* level index (0 = lowest) of t on odd-integer levels -(mq-1)..(mq-1);
 * thresholds at the even integers between them, ties to the upper level */
static int decide_dim(double t, int mq)
{
    int L = 0;
    for (int j = 0; j < mq - 1; j++)
        if (t >= (double)(2 * j - (mq - 2))) L = j + 1;
    return L;
}
static double level_value(int L, int mq) { return (double)(2 * L - (mq - 1)); }
static int near_dim(double t, int mq)
{
    for (int j = 0; j < mq - 1; j++)
        if (fabs(t - (double)(2 * j - (mq - 2))) < 1e-4) return 1;
    return 0;
}
/* squared distance of t to the nearest level */
static double dist_dim(double t, int mq)
{
    double best = INFINITY;
    for (int L = 0; L < mq; L++) {
        double d = t - level_value(L, mq);
        if (d * d < best) best = d * d;
    }
    return best;
}
static int gray_of(int L) { return L ^ (L >> 1); }
static int gray_inv(int g) { int L = g; for (int s = g >> 1; s; s >>= 1) L ^= s; return L; }
/* Differential quadrant coding (KK option, reading): the quadrant of a decided QAM
 * point (0: I > 0, Q > 0, then counterclockwise) and the point turned back into the
 * first quadrant, whose coordinates (1 + 2 b2, 1 + 2 b3) give the last two bits (16QAM) */
static int quad_of(int LI, int LQ, int mq, int *b2, int *b3)
{
    int I = 2 * LI - (mq - 1), Q = 2 * LQ - (mq - 1), q, x, y;
    if (I > 0 && Q > 0) { q = 0; x = I; y = Q; }
    else if (I < 0 && Q > 0) { q = 1; x = Q; y = -I; }
    else if (I < 0 && Q < 0) { q = 2; x = -I; y = -Q; }
    else { q = 3; x = -Q; y = I; }
    *b2 = (x - 1) / 2;
    *b3 = (y - 1) / 2;
    return q;
}

/* transmitted level indices of symbol k from the PRBS (MSB first) */
static void tx_symbol(const orx *h, int64_t k, int *LI, int *LQ)
{
    int nb = h->kk ? h->bps / 2 : h->bps;
    int64_t b0 = (int64_t)h->bps * k;
    int gi = 0, gq = 0;
    for (int t = 0; t < nb; t++) gi = (gi << 1) | h->prbs[(b0 + t) % 32767];
    if (h->kk)
        for (int t = 0; t < nb; t++) gq = (gq << 1) | h->prbs[(b0 + nb + t) % 32767];
    *LI = gray_inv(gi);
    *LQ = h->kk ? gray_inv(gq) : 0;
}

/* Blind-phase-search metric of one window (exported for the pins):
 * metric[b] = sum_k min_d |s z_k e^{-j theta_b} - d|^2, theta_b = (b/B)(pi/2) - pi/4,
 * d over the square constellation with mq odd-integer levels per dimension. */
void orx_bps_metrics(const double *z_re, const double *z_im, int W, int mq, double s, int B, double *metric)
{
    for (int b = 0; b < B; b++) {
        double tb = ((double)b / (double)B) * (PI / 2.0) - PI / 4.0;
        cx rot = cx_expj(-tb);
        double M = 0.0;
        for (int q = 0; q < W; q++) {
            cx t = cx_scale(cx_mul(cx_mk(z_re[q], z_im[q]), rot), s);
            M += dist_dim(t.re, mq) + dist_dim(t.im, mq);
        }
        metric[b] = M;
    }
}

/* ------------------------------------------------------------ call context */
typedef struct {
    orx *h;
    const int32_t *cur; int64_t base;   /* current buffer: stream samples [base, base+Nb) */
    cx *E; int64_t E_start, E_len;      /* this call's KK outputs */
    cx *y; int64_t y_start, y_len;      /* this call's matched-filter outputs */
    cx *R; int64_t R_start, R_len;      /* this call's resampled field (transmitter grid) */
    double mu_pam, sd_pam;
} ctx;

/* a read before the history a call keeps, or past what the call has computed, is a
 * bug of this program: stop loudly */
static void history_miss(const char *what, int64_t idx, int64_t start)
{
    fprintf(stderr, "rx_oracle: %s index %lld precedes the kept history (from %lld)\n", what, (long long)idx,
            (long long)start);
    abort();
}
static void past_end(const char *what, int64_t idx, int64_t end)
{
    fprintf(stderr, "rx_oracle: %s index %lld is past the computed values (to %lld)\n", what, (long long)idx,
            (long long)end);
    abort();
}
static int32_t code_at(const ctx *x, int64_t n)
{
    const orx *h = x->h;
    if (n < 0) return h->have_first ? h->first_code : x->cur[0];   /* pre-stream: first sample replicated */
    if (n >= x->base) return x->cur[n - x->base];
    int64_t i = n - (x->base - h->chist_len);
    if (i < 0) history_miss("12-bit code", n, x->base - h->chist_len);
    return h->chist[i];
}
static cx e_at(const ctx *x, int64_t n)
{
    const orx *h = x->h;
    if (n < 0) return cx_mk(0.0, 0.0);
    if (n >= x->E_start) {
        if (n >= x->E_start + x->E_len) past_end("field", n, x->E_start + x->E_len);
        return x->E[n - x->E_start];
    }
    if (n < h->ehist_start) history_miss("field", n, h->ehist_start);
    return h->ehist[n - h->ehist_start];
}
static cx r_at(const ctx *x, int64_t m)   /* the field on the grid the filter reads */
{
    const orx *h = x->h;
    if (!h->rs) return e_at(x, m);
    if (m < 0) return cx_mk(0.0, 0.0);
    if (m >= x->R_start) {
        if (m >= x->R_start + x->R_len) past_end("resampled field", m, x->R_start + x->R_len);
        return x->R[m - x->R_start];
    }
    if (m < h->rhist_start) history_miss("resampled field", m, h->rhist_start);
    return h->rhist[m - h->rhist_start];
}
static cx y_at(const ctx *x, int64_t m)
{
    const orx *h = x->h;
    if (m < 0) return cx_mk(0.0, 0.0);
    if (m >= x->y_start) {
        if (m >= x->y_start + x->y_len) past_end("2-sps sample", m, x->y_start + x->y_len);
        return x->y[m - x->y_start];
    }
    if (m < h->yhist_start) history_miss("2-sps sample", m, h->yhist_start);
    return h->yhist[m - h->yhist_start];
}

/* ------------------------------------------------ symbol-by-symbol DD-LMS (KK)
 * The paper's KK equaliser (Sec. 2, KK chain): a short decision-directed LMS
 * whose complex taps are updated after every symbol, so that they follow the
 * clock phase (a fractional delay at 2 samples/symbol) and the symbol phase (a
 * common rotation) together, with no separate phase search.  For symbols
 * k0 .. k0+n-1, with th = (ntaps-1)/2:
 *   z_k = sum_{j=0}^{ntaps-1} conj(w_j) y[2k + th - j]
 *   decision per dimension on s z_k
 *   error: CMA e = z (R2 - |z|^2) for k < cma_until (mu_cma), else
 *          decision-directed e = d/s - z (mu)
 *   then at once w_j += mu y[2k + th - j] conj(e). */
static void dd_symbols(ctx *x, cx *w, int64_t k0, int64_t n, int64_t cma_until, double mu_cma, double mu,
                       cx *z, cx *v, int32_t *draw, int32_t *nearf)
{
    orx *h = x->h;
    int nt = h->c.ntaps, th = h->th;
    for (int64_t q = 0; q < n; q++) {
        int64_t k = k0 + q;
        cx acc = cx_mk(0.0, 0.0);
        for (int j = 0; j < nt; j++) acc = cx_add(acc, cx_mul(cx_conj(w[j]), y_at(x, 2 * k + th - j)));
        z[q] = acc;
        cx t = cx_scale(acc, h->scale);
        v[q] = t;
        int LI = decide_dim(t.re, h->mq), LQ = decide_dim(t.im, h->mq);
        draw[2 * q] = LI; draw[2 * q + 1] = LQ;
        nearf[q] = near_dim(t.re, h->mq) || near_dim(t.im, h->mq);
        cx e;
        double m;
        if (k < cma_until) {
            e = cx_scale(acc, h->r2 - cx_abs2(acc));
            m = mu_cma;
        } else {
            cx d = cx_mk(level_value(LI, h->mq), level_value(LQ, h->mq));
            e = cx_sub(cx_scale(d, 1.0 / h->scale), acc);
            m = mu;
        }
        for (int j = 0; j < nt; j++)
            w[j] = cx_add(w[j], cx_scale(cx_mul(y_at(x, 2 * k + th - j), cx_conj(e)), m));
    }
}

/* ----------------------------------------------------------- equaliser window
 * One window of `win` symbols starting at symbol k0 with taps w:
 *   z_k = sum_i conj(w_i) y[2k - i]              (i = -th..th)
 *   blind phase search (decision-directed QAM): theta_b = (b/B)(pi/2) - pi/4,
 *   metric_b = sum_k min_d |s z_k e^{-j theta_b} - d|^2, b* = first argmin
 *   decision per dimension on s z_k e^{-j theta*}
 *   error: CMA  e = z (R2 - |z|^2);  data-aided  e = a_k - z;
 *          decision-directed  e = (d/s) e^{j theta*} - z
 *   block-LMS update after the window: w_i += mu sum_k y[2k-i] conj(e_k)
 * mode: 0 CMA, 1 data-aided, 2 decision-directed. */
typedef struct { int b; double best, second; } winres;

static winres eq_window(ctx *x, cx *w, int64_t k0, int mode, double mu,
                        cx *z, cx *v, int32_t *draw, int32_t *nearf, cx *grad)
{
    orx *h = x->h;
    int W = h->c.win, th = h->th;
    winres R; R.b = -1; R.best = 0.0; R.second = 0.0;
    for (int q = 0; q < W; q++) {
        int64_t k = k0 + q;
        cx acc = cx_mk(0.0, 0.0);
        for (int i = -th; i <= th; i++) acc = cx_add(acc, cx_mul(cx_conj(w[i + th]), y_at(x, 2 * k - i)));
        z[q] = acc;
    }
    double theta = 0.0;
    if (h->kk && mode == 2) {
        int B = h->c.bps_b;
        double best = INFINITY, second = INFINITY;
        int bb = 0;
        for (int b = 0; b < B; b++) {
            double tb = ((double)b / (double)B) * (PI / 2.0) - PI / 4.0;
            cx rot = cx_expj(-tb);
            double M = 0.0;
            for (int q = 0; q < W; q++) {
                cx t = cx_scale(cx_mul(z[q], rot), h->scale);
                M += dist_dim(t.re, h->mq) + dist_dim(t.im, h->mq);
            }
            if (M < best) { second = best; best = M; bb = b; }
            else if (M < second) second = M;
        }
        R.b = bb; R.best = best; R.second = second;
        theta = ((double)bb / (double)B) * (PI / 2.0) - PI / 4.0;
    }
    cx e[4096];
    cx rot = cx_expj(-theta), unrot = cx_expj(theta);
    for (int q = 0; q < W; q++) {
        int64_t k = k0 + q;
        cx t = cx_scale(cx_mul(z[q], rot), h->scale);
        v[q] = t;
        int LI = decide_dim(t.re, h->mq);
        int LQ = h->kk ? decide_dim(t.im, h->mq) : 0;
        draw[2 * q] = LI; draw[2 * q + 1] = LQ;
        nearf[q] = near_dim(t.re, h->mq) || (h->kk && near_dim(t.im, h->mq));
        if (mode == 0) {
            e[q] = cx_scale(z[q], h->r2 - cx_abs2(z[q]));
        } else if (mode == 1) {
            int aI, aQ;
            tx_symbol(h, k, &aI, &aQ);
            e[q] = cx_sub(cx_mk(level_value(aI, h->mq), 0.0), z[q]);
        } else {
            cx d = cx_mk(level_value(LI, h->mq), h->kk ? level_value(LQ, h->mq) : 0.0);
            e[q] = cx_sub(cx_mul(cx_scale(d, 1.0 / h->scale), unrot), z[q]);
        }
    }
    for (int i = -th; i <= th; i++) {
        cx g = cx_mk(0.0, 0.0);
        for (int q = 0; q < W; q++) g = cx_add(g, cx_mul(y_at(x, 2 * (k0 + q) - i), cx_conj(e[q])));
        if (grad) grad[i + th] = cx_add(grad[i + th], g);   /* frozen taps: gradient only */
        else w[i + th] = cx_add(w[i + th], cx_scale(g, mu));
    }
    return R;
}

static void put_bit(uint8_t *out, int64_t t, int bit)
{
    if (bit) out[t >> 3] |= (uint8_t)(0x80u >> (t & 7));
}

/* resampler accumulator at nominal sample m (>= rs_r0), in units of 2^-32 ADC samples */
static __int128 rs_psi(const orx *h, int64_t m) { return h->rs_psi0 + (__int128)(m - h->rs_r0) * h->rs_step; }
/* #{m >= 0 : accumulator(m) < lim}, for lim at or beyond the accumulator at rs_r0 */
static int64_t rs_below(const orx *h, __int128 lim)
{
    __int128 d = lim - h->rs_psi0;
    if (d <= 0) return h->rs_r0;
    return h->rs_r0 + (int64_t)((d + h->rs_step - 1) / h->rs_step);
}

/* Clock tracker (frequency-domain form): the block delays d_b = -(P / 2 pi) arg C_b of
 * every call, unwrapped against the last block of the previous call (period P = sps
 * samples, as within a call), feed least-squares sums over the blocks since the last
 * reset; x is the block centre (N/2) b + N/4 relative to the first block's. */
static void clock_track(orx *h, const cx *C, int64_t b0, int64_t nblk, int N, int sps)
{
    const double P = (double)sps, H = 0.5 * P;
    for (int64_t i = 0; i < nblk; i++) {
        double d = -P / (2.0 * PI) * atan2(C[i].im, C[i].re);
        double off = h->ck_have ? h->ck_off : 0.0;
        if (h->ck_have) {
            if (d + off - h->ck_y > H) off -= P;
            else if (d + off - h->ck_y < -H) off += P;
        }
        double y = d + off, c = (double)(N / 2) * (double)(b0 + i) + (double)(N / 4);
        if (h->ck_n == 0) h->ck_x0 = c;
        double x = c - h->ck_x0;
        h->ck_sx += x; h->ck_sy += y; h->ck_sxx += x * x; h->ck_sxy += x * y; h->ck_n++;
        h->ck_y = y; h->ck_off = off; h->ck_have = 1;
    }
}

/* One buffer through the chain.  `flush` marks a pad buffer of the stream end
 * (orx_flush): the carrier and gain (KK) or mean and deviation (PAM) stay those
 * of the last real buffer, and windows reaching symbol score_end are decided but
 * not scored. */
static int64_t process_buffer(orx *h, const uint8_t *packed, uint8_t *bits_out, int64_t bits_cap, int flush,
                              int64_t score_end)
{
    const orx_cfg *c = &h->c;
    int64_t Nb = c->buf_len;
    int32_t *cur = xcalloc((size_t)Nb, sizeof(int32_t));
    orx_unpack(packed, Nb, c->pack_order, cur);
    ctx X; memset(&X, 0, sizeof X);
    X.h = h; X.cur = cur; X.base = h->calls * Nb;
    if (!h->have_first) { h->first_code = cur[0]; h->have_first = 1; }
    int64_t avail = X.base + Nb;

    /* emission counts: every step emits what its full support allows */
    int64_t e_k = h->kk ? avail - c->ols_v / 2 : avail;
    if (e_k < 0) e_k = 0;
    /* resampler: nominal sample m needs the ADC field up to index i_m + 8, with
     * i_m = floor((rs_phase0 + m rs_step) / 2^32): r_k = #{m >= 0 : i_m + 8 < e_k} */
    int64_t r_k = e_k;
    if (h->rs) {
        r_k = rs_below(h, (__int128)(e_k - 8) << 32);
        if (r_k < h->r_prev) r_k = h->r_prev;
    }
    int64_t f_k = (r_k >= h->hmf + 1) ? (r_k - h->hmf - 1) / h->dec + 1 : 0;
    if (h->fd) {   /* whole blocks: block b needs the inputs up to hop*b + 3N/4 */
        int64_t N = c->fd_n, hop = N / 2;
        int64_t bk = (r_k >= 3 * N / 4) ? (r_k - 3 * N / 4) / hop + 1 : 0;
        f_k = bk * (hop / h->dec);
    }
    int64_t s_k = (f_k >= h->th + 1) ? (f_k - h->th - 1) / 2 + 1 : 0;
    int64_t q_k = (s_k >= c->ntrain) ? c->ntrain + ((s_k - c->ntrain) / c->eq_block) * c->eq_block : 0;
    if (q_k < h->q_prev) q_k = h->q_prev;

    /* ---- KK field reconstruction by overlap-save blocks ---------------- */
    X.E_start = h->e_prev; X.E_len = h->kk ? e_k - h->e_prev : 0;
    X.E = xcalloc((size_t)(X.E_len > 0 ? X.E_len : 1), sizeof(cx));
    if (h->kk && X.E_len > 0) {
        int N = c->ols_n, V = c->ols_v, hop = N - V;
        double *u = xcalloc((size_t)N, sizeof(double)), *phi = xcalloc((size_t)N, sizeof(double));
        double *re = xcalloc((size_t)N, sizeof(double)), *im = xcalloc((size_t)N, sizeof(double));
        int64_t J = (X.E_len + hop - 1) / hop;
        for (int64_t j = 0; j < J; j++) {
            int64_t o = h->e_prev + j * hop;                   /* first kept output */
            int64_t ws = (j < J - 1) ? o - V / 2 : avail - N;   /* last block ends at the newest sample */
            int64_t cnt = (j < J - 1) ? hop : e_k - o;
            for (int t = 0; t < N; t++) u[t] = 0.5 * log(kk_intensity(code_at(&X, ws + t)));
            hilbert_block(u, phi, N, re, im);
            for (int64_t n = o; n < o + cnt; n++) {
                double a = sqrt(kk_intensity(code_at(&X, n)));
                X.E[n - X.E_start] = cx_scale(cx_expj(phi[n - ws]), a);
            }
        }
        free(u); free(phi); free(re); free(im);
        /* carrier (the real tone of the KK field) and signal-power gain of this call:
         * c = mean E, P = mean I - |c|^2, g = 1/sqrt(sps P)  (reading) */
        cx sumE = cx_mk(0.0, 0.0);
        double sumI = 0.0;
        for (int64_t n = h->e_prev; n < e_k; n++) {
            sumE = cx_add(sumE, X.E[n - X.E_start]);
            sumI += kk_intensity(code_at(&X, n));
        }
        if (!flush) {
            h->carrier = cx_scale(sumE, 1.0 / (double)X.E_len);
            double P = sumI / (double)X.E_len - cx_abs2(h->carrier);
            h->gain = (P > 0.0) ? 1.0 / sqrt((double)c->sps * P) : 1.0;
        }
    }
    if (!h->kk) {
        /* DC removal and scaling by the buffer's mean and standard deviation */
        double s1 = 0.0, s2 = 0.0;
        for (int64_t i = 0; i < Nb; i++) { s1 += cur[i]; s2 += (double)cur[i] * cur[i]; }
        X.mu_pam = s1 / (double)Nb;
        double var = s2 / (double)Nb - X.mu_pam * X.mu_pam;
        X.sd_pam = (var > 0.0) ? sqrt(var) : 1.0;
        if (flush) { X.mu_pam = h->last_mu; X.sd_pam = h->last_sd; }
        h->last_mu = X.mu_pam; h->last_sd = X.sd_pam;
    }
    X.R_start = h->r_prev; X.R_len = h->rs ? r_k - h->r_prev : 0;
    X.R = xcalloc((size_t)(X.R_len > 0 ? X.R_len : 1), sizeof(cx));
    /* resampler to the transmitter's grid: KK interpolates the reconstructed field,
     * PAM the normalised code (zero before the stream), both computed in the call
     * that emits the nominal sample */
    for (int64_t m = h->r_prev; m < r_k && h->rs; m++) {
        __int128 psi = rs_psi(h, m);
        int64_t i = (int64_t)(psi >> 32);
        uint32_t fr = (uint32_t)(psi & 0xFFFFFFFF);
        double cj[16];
        orx_rs_taps((double)(fr >> 22) / 1024.0, cj);
        cx acc = cx_mk(0.0, 0.0);
        for (int j = -7; j <= 8; j++) {
            int64_t n = i + j;
            cx v = h->kk ? e_at(&X, n)
                         : cx_mk(n < 0 ? 0.0 : ((double)code_at(&X, n) - X.mu_pam) / X.sd_pam, 0.0);
            acc = cx_add(acc, cx_scale(v, cj[j + 7]));
        }
        X.R[m - X.R_start] = acc;
    }

    /* ---- matched filter (and 4 -> 2 samples/symbol for KK) ------------- */
    X.y_start = h->f_prev; X.y_len = f_k - h->f_prev;
    X.y = xcalloc((size_t)(X.y_len > 0 ? X.y_len : 1), sizeof(cx));
    if (h->fd && !h->kk) {
        /* PAM: static frequency-domain filter on N-point blocks with hop N/2 at the
         * input rate; the block input is the normalised code, zero before the stream */
        int N = c->fd_n, hop = N / 2;
        free(h->d_C);
        h->d_C_start = h->f_prev / hop;
        h->d_C_len = f_k / hop - h->d_C_start;
        h->d_C = xcalloc((size_t)(h->d_C_len > 0 ? h->d_C_len : 1), sizeof(cx));
        double *xr = xcalloc((size_t)N, sizeof(double)), *xi = xcalloc((size_t)N, sizeof(double));
        double *yr = xcalloc((size_t)(N / 2), sizeof(double)), *yi = xcalloc((size_t)(N / 2), sizeof(double));
        for (int64_t b = h->f_prev / hop; b < f_k / hop; b++) {
            for (int t = 0; t < N; t++) {
                int64_t n = (int64_t)hop * b - N / 4 + t;
                xr[t] = n < 0 ? 0.0 : ((double)code_at(&X, n) - X.mu_pam) / X.sd_pam;
                xi[t] = 0.0;
            }
            orx_fd_block_full(xr, xi, N, h->fd_Hr, h->fd_Hi, yr, yi);
            {
                int w = (int)ceil(c->rrc_beta * N / 4.0);   /* ceil(beta S / 2), S = N / 2 */
                double cr, ci;
                orx_fd_clock(xr, xi, N, h->fd_Hr, h->fd_Hi, 2, w, &cr, &ci);
                h->d_C[b - h->d_C_start] = cx_mk(cr, ci);
            }
            for (int m = 0; m < N / 2; m++) X.y[(int64_t)hop * b + m - X.y_start] = cx_mk(yr[m], 0.0);
        }
        free(xr); free(xi); free(yr); free(yi);
        if (c->clk_track) clock_track(h, h->d_C, h->d_C_start, h->d_C_len, N, 2);
    } else if (h->fd) {
        /* static frequency-domain filter, N-point blocks with hop N/2, bin-truncation
         * downsampling; the block input is the carrier-removed, downshifted field */
        int N = c->fd_n, hop = N / 2;
        free(h->d_C);
        h->d_C_start = h->f_prev / (hop / 2);
        h->d_C_len = f_k / (hop / 2) - h->d_C_start;
        h->d_C = xcalloc((size_t)(h->d_C_len > 0 ? h->d_C_len : 1), sizeof(cx));
        double *xr = xcalloc((size_t)N, sizeof(double)), *xi = xcalloc((size_t)N, sizeof(double));
        double *yr = xcalloc((size_t)(N / 4), sizeof(double)), *yi = xcalloc((size_t)(N / 4), sizeof(double));
        for (int64_t b = h->f_prev / (hop / 2); b < f_k / (hop / 2); b++) {
            for (int t = 0; t < N; t++) {
                int64_t n = (int64_t)hop * b - N / 4 + t;
                cx xn = cx_mk(0.0, 0.0);
                if (n >= 0) {
                    int64_t p = ((n % c->ds_den) * c->ds_num) % c->ds_den;
                    xn = cx_mul(cx_sub(r_at(&X, n), h->carrier), cx_expj(-2.0 * PI * (double)p / (double)c->ds_den));
                }
                xr[t] = xn.re; xi[t] = xn.im;
            }
            orx_fd_block(xr, xi, N, h->fd_Hr, h->fd_Hi, yr, yi);
            {
                int w = (int)ceil(c->rrc_beta * N / 8.0);   /* ceil(beta S / 2), S = N / 4 */
                double cr, ci;
                orx_fd_clock(xr, xi, N, h->fd_Hr, h->fd_Hi, 4, w, &cr, &ci);
                h->d_C[b - h->d_C_start] = cx_mk(cr, ci);
            }
            for (int m = 0; m < N / 4; m++)
                X.y[(int64_t)(hop / 2) * b + m - X.y_start] = cx_scale(cx_mk(yr[m], yi[m]), h->gain);
        }
        free(xr); free(xi); free(yr); free(yi);
        if (c->clk_track) clock_track(h, h->d_C, h->d_C_start, h->d_C_len, N, 4);
    }
    for (int64_t m = h->fd ? f_k : h->f_prev; m < f_k; m++) {
        cx acc = cx_mk(0.0, 0.0);
        for (int i = -h->hmf; i <= h->hmf; i++) {
            int64_t n = (int64_t)h->dec * m - i;
            if (n < 0) continue;
            cx xn;
            if (h->kk) {
                /* carrier removal, then downshift by ds_num/ds_den cycles/sample */
                int64_t p = ((n % c->ds_den) * c->ds_num) % c->ds_den;
                xn = cx_mul(cx_sub(r_at(&X, n), h->carrier),
                            cx_expj(-2.0 * PI * (double)p / (double)c->ds_den));
            } else if (h->rs) {
                xn = r_at(&X, n);
            } else {
                xn = cx_mk(((double)code_at(&X, n) - X.mu_pam) / X.sd_pam, 0.0);
            }
            acc = cx_add(acc, cx_scale(xn, h->rrc[i + h->hmf]));
        }
        X.y[m - X.y_start] = h->kk ? cx_scale(acc, h->gain) : acc;
    }

    /* ---- equaliser ------------------------------------------------------ */
    int W = c->win;
    int64_t sym_lo = h->trained ? h->q_prev : 0;
    int64_t nproc = (q_k > sym_lo) ? q_k - sym_lo : 0;
    if (!h->trained && q_k < c->ntrain) nproc = 0;
    cx *Z = xcalloc((size_t)(nproc + 1), sizeof(cx)), *Vv = xcalloc((size_t)(nproc + 1), sizeof(cx));
    int32_t *draw = xcalloc((size_t)(2 * nproc + 2), sizeof(int32_t));
    int32_t *nearf = xcalloc((size_t)(nproc + 1), sizeof(int32_t));
    int64_t pay_lo = sym_lo;
    if (nproc > 0 && !h->trained) {
        /* training at stream start, sequential over windows: KK CMA for the first
         * ncma symbols then decision-directed; PAM data-aided LMS */
        if (c->eq_mode == 1) {
            dd_symbols(&X, h->w, 0, c->ntrain, c->ncma, c->mu_cma, c->mu, Z, Vv, draw, nearf);
        } else {
            for (int64_t k0 = 0; k0 < c->ntrain; k0 += W) {
                int mode = h->kk ? (k0 < c->ncma ? 0 : 2) : 1;
                double mu = h->kk ? (mode == 0 ? c->mu_cma : c->mu) : c->mu_train;
                eq_window(&X, h->w, k0, mode, mu, Z + k0, Vv + k0, draw + 2 * k0, nearf + k0, NULL);
            }
        }
        h->trained = 1;
        pay_lo = c->ntrain;
    }
    int64_t npay = (nproc > 0) ? q_k - pay_lo : 0;
    int64_t nwin = npay / W;
    double *dwin = xcalloc((size_t)(4 * nwin + 4), sizeof(double));
    int64_t *msym = xcalloc((size_t)(npay + 1), sizeof(int64_t));
    if (npay > 0) {
        /* payload: independent blocks of eq_block symbols, all starting from the
         * same taps (block parallelism of the 8192 data blocks, Sec. 2) */
        cx *wb = xcalloc((size_t)c->ntaps, sizeof(cx)), *wlast = xcalloc((size_t)c->ntaps, sizeof(cx));
        /* frozen taps (eq_frozen, KK, reading of the block-Toeplitz form): every
         * symbol of a block is filtered with the taps the call started from, so
         * the filter of the whole call is one fixed FIR; the gradient of the last
         * block, sum_k y[2k-i] conj(e_k), is summed window by window, and the next
         * call starts from w + mu (W / eq_block) times it, i.e. the mean of the
         * block's per-window steps */
        int frozen = h->kk && c->eq_frozen;
        cx *gsum = xcalloc((size_t)c->ntaps, sizeof(cx)), *gdrop = xcalloc((size_t)c->ntaps, sizeof(cx));
        for (int64_t b0 = pay_lo; b0 < q_k; b0 += c->eq_block) {
            memcpy(wb, h->w, sizeof(cx) * (size_t)c->ntaps);
            int last = b0 + c->eq_block >= q_k;
            if (c->eq_mode == 1) {
                /* symbol-by-symbol DD-LMS: no phase search, window index 0 throughout */
                int64_t o = b0 - sym_lo;
                dd_symbols(&X, wb, b0, c->eq_block, -1, 0.0, c->mu, Z + o, Vv + o, draw + 2 * o, nearf + o);
                memcpy(wlast, wb, sizeof(cx) * (size_t)c->ntaps);
                continue;
            }
            for (int64_t k0 = b0; k0 < b0 + c->eq_block; k0 += W) {
                int64_t o = k0 - sym_lo;
                winres R = eq_window(&X, wb, k0, 2, c->mu, Z + o, Vv + o, draw + 2 * o, nearf + o,
                                     frozen ? (last ? gsum : gdrop) : NULL);
                int64_t wi = (k0 - pay_lo) / W;
                dwin[4 * wi] = R.b; dwin[4 * wi + 2] = R.best; dwin[4 * wi + 3] = R.second;
                if (h->kk && (R.second - R.best) <= 1e-6 * R.best) h->n_amb++;
            }
            if (!frozen) memcpy(wlast, wb, sizeof(cx) * (size_t)c->ntaps);
        }
        if (frozen) {
            double step = c->mu * (double)W / (double)c->eq_block;
            for (int i = 0; i < c->ntaps; i++) h->w[i] = cx_add(h->w[i], cx_scale(gsum[i], step));
        } else {
            memcpy(h->w, wlast, sizeof(cx) * (size_t)c->ntaps);
        }
        free(wb); free(wlast); free(gsum); free(gdrop);
        /* integer pi/2 unwrap of the window phase index, carried across calls */
        for (int64_t wi = 0; wi < nwin; wi++) {
            int b = (int)dwin[4 * wi];
            int64_t m = 0;
            if (h->kk) {
                if (h->have_b) {
                    int d = h->b_last - b;
                    m = h->m_last + (d > c->bps_b / 2) - (d < -c->bps_b / 2);
                }
                h->have_b = 1; h->b_last = b; h->m_last = m;
            }
            dwin[4 * wi + 1] = (double)m;
            for (int q = 0; q < W; q++) msym[wi * W + q] = m;
        }
        h->n_win += nwin;
    }

    /* ---- ambiguity, demap, bit errors ---------------------------------- */
    int32_t *ahat = xcalloc((size_t)(2 * nproc + 2), sizeof(int32_t));
    int32_t *berr = xcalloc((size_t)(nproc + 1), sizeof(int32_t));
    for (int64_t i = 0; i < nproc; i++) { ahat[2 * i] = draw[2 * i]; ahat[2 * i + 1] = draw[2 * i + 1]; berr[i] = -1; }
    int64_t off = pay_lo - sym_lo;
    if (h->kk && npay > 0 && !h->amb_done) {
        /* resolve the pi/2 ambiguity once: the rotation whose first amb_syms
         * payload decisions best match the known transmitted symbols (reading) */
        int64_t A = c->amb_syms < npay ? c->amb_syms : npay;
        int best_r = 0; int64_t best_cnt = -1;
        for (int r = 0; r < 4; r++) {
            int64_t cnt = 0;
            for (int64_t i = 0; i < A; i++) {
                int LI = draw[2 * (off + i)], LQ = draw[2 * (off + i) + 1];
                int q = (int)(((msym[i] + r) % 4 + 4) % 4);
                for (int s = 0; s < q; s++) { int t = LI; LI = LQ; LQ = h->mq - 1 - t; }
                int aI, aQ;
                tx_symbol(h, pay_lo + i, &aI, &aQ);
                cnt += (LI != aI || LQ != aQ);
            }
            if (best_cnt < 0 || cnt < best_cnt) { best_cnt = cnt; best_r = r; }
        }
        h->amb_r = best_r; h->amb_done = 1;
    }
    int64_t nbits = (int64_t)h->bps * npay;
    if (bits_out && bits_cap > 0) memset(bits_out, 0, (size_t)((bits_cap + 7) / 8));
    int32_t *dword = xcalloc((size_t)(nproc + 1), sizeof(int32_t));   /* differentially decoded words */
    int nb = h->kk ? h->bps / 2 : h->bps;
    for (int64_t i = 0; i < npay; i++) {
        int64_t o = off + i;
        int LI = draw[2 * o], LQ = draw[2 * o + 1];
        if (h->kk) {
            int q = (int)(((msym[i] + h->amb_r) % 4 + 4) % 4);
            for (int s = 0; s < q; s++) { int t = LI; LI = LQ; LQ = h->mq - 1 - t; }
        }
        ahat[2 * o] = LI; ahat[2 * o + 1] = LQ;
        int gi = gray_of(LI), gq = gray_of(LQ);
        int64_t t0 = (int64_t)h->bps * i;
        if (h->kk && c->diff_code) {
            /* differential decoding: the quadrant step from the previous symbol (Gray),
             * then the point's bits in its quadrant; the word replaces (gi, gq) */
            int b2, b3, q = quad_of(LI, LQ, h->mq, &b2, &b3);
            int d = ((q - (h->dq_have ? h->dq_prev : q)) % 4 + 4) % 4, gd = d ^ (d >> 1);
            int w = (h->mq == 4) ? (gd << 2) | (b2 << 1) | b3 : gd;
            dword[o] = w;
            h->dq_prev = q; h->dq_have = 1;
            if (bits_out && t0 + h->bps <= bits_cap)
                for (int t = 0; t < h->bps; t++) put_bit(bits_out, t0 + t, (w >> (h->bps - 1 - t)) & 1);
            continue;
        }
        if (bits_out && t0 + h->bps <= bits_cap) {
            for (int t = 0; t < nb; t++) put_bit(bits_out, t0 + t, (gi >> (nb - 1 - t)) & 1);
            if (h->kk) for (int t = 0; t < nb; t++) put_bit(bits_out, t0 + nb + t, (gq >> (nb - 1 - t)) & 1);
        }
    }
    /* Bit-error counting against the PRBS, window by window.  The blind phase
     * search holds one phase per window, so a cycle slip can only start at a
     * window edge; like a BER tester that re-synchronises after a slip, each
     * window is scored under the pi/2 rotation (applied on top of the decoded
     * symbols) with the fewest bit errors, ties to no rotation (reading).  PAM
     * has no rotation.  Symbols used to resolve the stream-start ambiguity are
     * not counted. */
    for (int64_t wi = 0; wi < nwin; wi++) {
        int64_t k0 = pay_lo + wi * W;
        if (h->kk && k0 < c->ntrain + c->amb_syms) continue;
        if (k0 + W > score_end) continue;   /* stream end: filter supports reach into the pad */
        if (h->kk && c->diff_code) {
            /* the decoded data bits against the PRBS: rotation-free, so one count serves
             * both the BER-tester view and the delivered output */
            for (int q = 0; q < W; q++) {
                int64_t o = off + wi * W + q, k = k0 + q;
                int ne = 0;
                for (int t = 0; t < h->bps; t++)
                    ne += ((dword[o] >> (h->bps - 1 - t)) & 1) != h->prbs[((int64_t)h->bps * k + t) % 32767];
                berr[o] = ne;
                h->n_bit_err += ne;
                h->n_raw_err += ne;
                h->n_sym_err += ne > 0;
                h->n_near += nearf[o];
            }
            h->n_bits += (int64_t)h->bps * W;
            h->n_symbols += W;
            continue;
        }
        int nrot = h->kk ? 4 : 1;
        int64_t errs[4] = {0, 0, 0, 0};
        for (int rho = 0; rho < nrot; rho++) {
            for (int q = 0; q < W; q++) {
                int64_t o = off + wi * W + q, k = k0 + q;
                int LI = ahat[2 * o], LQ = ahat[2 * o + 1];
                for (int s = 0; s < rho; s++) { int t = LI; LI = LQ; LQ = h->mq - 1 - t; }
                int gi = gray_of(LI), gq = gray_of(LQ), bitsym[8];
                for (int t = 0; t < nb; t++) bitsym[t] = (gi >> (nb - 1 - t)) & 1;
                if (h->kk) for (int t = 0; t < nb; t++) bitsym[nb + t] = (gq >> (nb - 1 - t)) & 1;
                int ne = 0;
                for (int t = 0; t < h->bps; t++) ne += bitsym[t] != h->prbs[((int64_t)h->bps * k + t) % 32767];
                errs[rho] += ne;
                if (rho == 0) berr[o] = ne;
            }
        }
        int best = 0;
        for (int rho = 1; rho < nrot; rho++) if (errs[rho] < errs[best]) best = rho;
        if (best != 0) {
            for (int q = 0; q < W; q++) {   /* per-symbol errors under the chosen rotation */
                int64_t o = off + wi * W + q, k = k0 + q;
                int LI = ahat[2 * o], LQ = ahat[2 * o + 1];
                for (int s = 0; s < best; s++) { int t = LI; LI = LQ; LQ = h->mq - 1 - t; }
                int gi = gray_of(LI), gq = gray_of(LQ), bitsym[8];
                for (int t = 0; t < nb; t++) bitsym[t] = (gi >> (nb - 1 - t)) & 1;
                if (h->kk) for (int t = 0; t < nb; t++) bitsym[nb + t] = (gq >> (nb - 1 - t)) & 1;
                int ne = 0;
                for (int t = 0; t < h->bps; t++) ne += bitsym[t] != h->prbs[((int64_t)h->bps * k + t) % 32767];
                berr[o] = ne;
            }
            h->n_slip++;
        }
        h->n_raw_err += errs[0];
        h->n_bit_err += errs[best];
        h->n_bits += (int64_t)h->bps * W;
        for (int q = 0; q < W; q++) {
            int64_t o = off + wi * W + q;
            h->n_sym_err += berr[o] > 0;
            h->n_near += nearf[o];
        }
        h->n_symbols += W;
    }

    /* ---- debug views ---------------------------------------------------- */
    free(h->d_E); free(h->d_y); free(h->d_z); free(h->d_v); free(h->d_ahat);
    free(h->d_draw); free(h->d_berr); free(h->d_near); free(h->d_win);
    h->d_E = X.E; h->d_E_start = X.E_start; h->d_E_len = X.E_len > 0 ? X.E_len : 0;
    free(h->d_R);
    h->d_R = X.R; h->d_R_start = X.R_start; h->d_R_len = X.R_len > 0 ? X.R_len : 0;
    h->d_y = X.y; h->d_y_start = X.y_start; h->d_y_len = X.y_len > 0 ? X.y_len : 0;
    h->d_z = Z; h->d_v = Vv; h->d_ahat = ahat; h->d_draw = draw; h->d_berr = berr; h->d_near = nearf;
    h->d_s_start = sym_lo; h->d_s_len = nproc;
    free(dword);
    h->d_win = dwin; h->d_win_len = nwin;
    h->scal[0] = h->carrier.re; h->scal[1] = h->carrier.im; h->scal[2] = h->gain;
    h->scal[3] = X.mu_pam; h->scal[4] = X.sd_pam;
    free(msym);

    /* ---- carry the stream state to the next buffer ----------------------- */
    if (h->rs && r_k > 0) {
        /* the filter's history on the transmitter grid */
        int64_t lo = h->fd ? (int64_t)h->dec * f_k - c->fd_n / 4 : (int64_t)h->dec * f_k - h->hmf;
        if (lo < 0) lo = 0;
        cx *nh = xcalloc((size_t)(r_k - lo + 1), sizeof(cx));
        for (int64_t m = lo; m < r_k; m++) nh[m - lo] = r_at(&X, m);
        free(h->rhist); h->rhist = nh; h->rhist_start = lo; h->rhist_len = r_k - lo;
    }
    if (h->kk && e_k > 0) {
        int64_t lo = h->fd ? (int64_t)h->dec * f_k - c->fd_n / 4 : (int64_t)h->dec * f_k - h->hmf;
        if (h->rs)   /* the resampler's next input: from i at nominal r_k, less 7, and less 4
                      * more for a re-timing between calls (its nudge is within half a symbol) */
            lo = (int64_t)(rs_psi(h, r_k) >> 32) - 11;
        if (lo < 0) lo = 0;
        if (lo > e_k) lo = e_k;
        cx *nh = xcalloc((size_t)(e_k - lo + 1), sizeof(cx));
        for (int64_t n = lo; n < e_k; n++) nh[n - lo] = e_at(&X, n);
        free(h->ehist); h->ehist = nh; h->ehist_start = lo; h->ehist_len = e_k - lo;
    }
    {
        /* the 2-sps history the next call's first symbols read: the filter of
         * symbol k reaches back to y[2k + th - (ntaps - 1)], ntaps - 1 - th samples
         * before 2k (th for the symmetric window filter; one more for an even tap
         * count of the symbol-by-symbol form) */
        int64_t lo = 2 * (h->trained ? q_k : 0) - (c->ntaps - 1 - h->th);
        if (lo < 0) lo = 0;
        if (lo > f_k) lo = f_k;
        cx *nh = xcalloc((size_t)(f_k - lo + 1), sizeof(cx));
        for (int64_t m = lo; m < f_k; m++) nh[m - lo] = y_at(&X, m);
        free(h->yhist); h->yhist = nh; h->yhist_start = lo; h->yhist_len = f_k - lo;
    }
    {
        int64_t keep = avail < h->chist_cap ? avail : h->chist_cap;
        int32_t *nh = xcalloc((size_t)h->chist_cap, sizeof(int32_t));
        for (int64_t i = 0; i < keep; i++) nh[i] = code_at(&X, avail - keep + i);
        free(h->chist); h->chist = nh; h->chist_len = keep;
    }
    h->e_prev = e_k; h->f_prev = f_k; h->q_prev = q_k; h->r_prev = r_k;
    h->calls++;
    if (!flush) h->n_samples += Nb;
    free(cur);
    return nbits;
}

int64_t orx_process(orx *h, const uint8_t *packed, uint8_t *bits_out, int64_t bits_cap)
{
    if (h->flushed) return -1;
    return process_buffer(h, packed, bits_out, bits_cap, 0, INT64_MAX);
}

/* End of the stream.  Every step emits only what its full support allows, so the
 * symbols of the last few thousand samples are still undecided after the last
 * buffer.  The stream is continued after its last sample with that sample's
 * code repeated (the mirror of the stream start, where the first sample is
 * replicated; reading), buffer by buffer, until every symbol whose centre lies
 * inside the stream (nominal sample k sps < the stream's nominal length) has been
 * decided.  Returns the bits of payload symbols [first undecided, last in the
 * stream]; windows whose last symbol lies within ceil((mf_span + ntaps) / 2)
 * symbols of the end are not scored. */
int64_t orx_flush(orx *h, uint8_t *bits_out, int64_t bits_cap)
{
    const orx_cfg *c = &h->c;
    if (bits_out && bits_cap > 0) memset(bits_out, 0, (size_t)((bits_cap + 7) / 8));
    if (h->flushed) return 0;
    h->flushed = 1;
    if (h->calls == 0) return 0;
    int64_t total = h->calls * c->buf_len, r_end = total;
    if (h->rs) r_end = rs_below(h, (__int128)total << 32);
    int64_t S = r_end > 0 ? (r_end - 1) / c->sps + 1 : 0;
    int64_t first = h->q_prev > c->ntrain ? h->q_prev : c->ntrain;
    if (S <= first) return 0;
    int32_t last = h->chist[h->chist_len - 1];
    int64_t nbytes = c->buf_len * 3 / 2;
    uint8_t *pad = xcalloc((size_t)nbytes, 1);
    for (int64_t i = 0; i < nbytes; i += 3) {   /* the pair (last, last) in the ADC word order */
        if (c->pack_order == 0) {
            pad[i] = (uint8_t)(last & 0xFF);
            pad[i + 1] = (uint8_t)(((last >> 8) & 0xF) | ((last & 0xF) << 4));
            pad[i + 2] = (uint8_t)(last >> 4);
        } else {
            pad[i] = (uint8_t)(last >> 4);
            pad[i + 1] = (uint8_t)(((last & 0xF) << 4) | ((last >> 8) & 0xF));
            pad[i + 2] = (uint8_t)(last & 0xFF);
        }
    }
    int64_t cap = (int64_t)h->bps * (c->buf_len + 8 * c->eq_block + c->ntrain + 65536);
    uint8_t *tmp = xcalloc((size_t)(cap / 8 + 1), 1);
    int64_t done = 0, score_end = S - (c->mf_span + c->ntaps + 1) / 2;
    while (h->q_prev < S) {
        int64_t q0 = h->q_prev;
        int trained = h->trained;
        int64_t nb = process_buffer(h, pad, tmp, cap, 1, score_end);
        h->pad_calls++;
        int64_t pay_lo = trained ? q0 : c->ntrain;
        int64_t hi = h->q_prev < S ? h->q_prev : S;
        for (int64_t t = 0; nb > 0 && t < (int64_t)h->bps * (hi - pay_lo); t++) {
            int bit = (tmp[t >> 3] >> (7 - (t & 7))) & 1;
            if (bits_out && done < bits_cap) put_bit(bits_out, done, bit);
            done++;
        }
    }
    free(pad); free(tmp);
    return done;
}

/* The tracker's line fit over the blocks since the last reset (the convention of
 * orx_clock_fit: d_b = -tau0 - eps c_b, c_b the block centre): ppm = 1e6 eps and the
 * delay at stream index 0, in (-sps/2, sps/2].  Returns the block count, -1 below 2. */
int64_t orx_clock_track(const orx *h, double *ppm, double *delay)
{
    if (h->ck_n < 2) return -1;
    const double P = (double)h->c.sps, H = 0.5 * P, nb = (double)h->ck_n;
    double slope = (nb * h->ck_sxy - h->ck_sx * h->ck_sy) / (nb * h->ck_sxx - h->ck_sx * h->ck_sx);
    double tau0 = -((h->ck_sy - slope * h->ck_sx) / nb - slope * h->ck_x0);
    while (tau0 > H) tau0 -= P;
    while (tau0 <= -H) tau0 += P;
    *ppm = -slope * 1e6;
    *delay = tau0;
    return h->ck_n;
}

/* New resampler accumulator from the next nominal sample r on: its ADC position moves
 * by `nudge` (2^-32 ADC samples) and later samples advance by `step`.  The tracker
 * restarts (sums and unwrap carry): later estimates are residuals against it. */
int orx_set_rs(orx *h, int64_t step, int64_t nudge)
{
    if (!h->rs || step < (int64_t)4252017623LL || step > (int64_t)4337916969LL) return -1;
    h->rs_psi0 = rs_psi(h, h->r_prev) + (__int128)nudge;
    h->rs_r0 = h->r_prev;
    h->rs_step = step;
    h->ck_n = 0; h->ck_sx = h->ck_sy = h->ck_sxx = h->ck_sxy = 0.0;
    h->ck_have = 0;
    return 0;
}

/* Closed loop (a second-order timing loop run between calls): the tracker's line
 * y(c) = y0 + s (c - x0) of the unwrapped block delays (the symbol grid sits at
 * resampled sample positions congruent to y mod P) re-times the accumulator from the
 * next nominal sample r: the grid drifts by s samples per sample, so the step scales
 * to round(step (1 + s)), and the grid is off by y(r) now, so the position moves by
 * round(w step) with w = y(r) wrapped into (-P/2, P/2] (whole symbols are not
 * observable and are left alone).  Halves round away from zero.  Returns 0, or -1 (no
 * resampler, fewer than 2 blocks, or a step outside 1 % of 2^32); *step_out and
 * *nudge_out receive the applied values. */
int orx_clock_retime(orx *h, int64_t *step_out, int64_t *nudge_out)
{
    if (!h->rs || h->ck_n < 2) return -1;
    const double P = (double)h->c.sps, H = 0.5 * P, nb = (double)h->ck_n;
    double s = (nb * h->ck_sxy - h->ck_sx * h->ck_sy) / (nb * h->ck_sxx - h->ck_sx * h->ck_sx);
    double y0 = (h->ck_sy - s * h->ck_sx) / nb;
    double w = y0 + s * ((double)h->r_prev - h->ck_x0);
    w -= P * floor(w / P);          /* [0, P) */
    if (w > H) w -= P;              /* (-P/2, P/2] */
    int64_t step = (int64_t)llround((double)h->rs_step * (1.0 + s));
    int64_t nudge = (int64_t)llround(w * (double)h->rs_step);
    if (orx_set_rs(h, step, nudge) != 0) return -1;
    if (step_out) *step_out = step;
    if (nudge_out) *nudge_out = nudge;
    return 0;
}

int64_t orx_get(orx *h, int what, void *dst, int64_t cap, int64_t *start)
{
    int64_t n = 0, s = 0, width = 0;
    const void *src = NULL;
    switch (what) {
    case ORX_E: n = h->d_E_len; s = h->d_E_start; src = h->d_E; width = sizeof(cx); break;
    case ORX_RS: n = h->d_R_len; s = h->d_R_start; src = h->d_R; width = sizeof(cx); break;
    case ORX_CLK: n = h->d_C_len; s = h->d_C_start; src = h->d_C; width = sizeof(cx); break;
    case ORX_Y: n = h->d_y_len; s = h->d_y_start; src = h->d_y; width = sizeof(cx); break;
    case ORX_Z: n = h->d_s_len; s = h->d_s_start; src = h->d_z; width = sizeof(cx); break;
    case ORX_V: n = h->d_s_len; s = h->d_s_start; src = h->d_v; width = sizeof(cx); break;
    case ORX_AHAT: n = h->d_s_len; s = h->d_s_start; src = h->d_ahat; width = 2 * sizeof(int32_t); break;
    case ORX_BERR: n = h->d_s_len; s = h->d_s_start; src = h->d_berr; width = sizeof(int32_t); break;
    case ORX_WIN: n = h->d_win_len; s = 0; src = h->d_win; width = 4 * sizeof(double); break;
    case ORX_TAPS: n = h->c.ntaps; s = 0; src = h->w; width = sizeof(cx); break;
    case ORX_SCAL: n = 5; s = 0; src = h->scal; width = sizeof(double); break;
    case ORX_NEAR: n = h->d_s_len; s = h->d_s_start; src = h->d_near; width = sizeof(int32_t); break;
    case ORX_DRAW: n = h->d_s_len; s = h->d_s_start; src = h->d_draw; width = 2 * sizeof(int32_t); break;
    default: return -1;
    }
    if (start) *start = s;
    if (dst && src && cap > 0) memcpy(dst, src, (size_t)((n < cap ? n : cap) * width));
    return n;
}

void orx_stats(orx *h, orx_stats_t *o)
{
    memset(o, 0, sizeof *o);
    o->calls = h->calls - h->pad_calls; o->samples = h->n_samples; o->symbols = h->n_symbols;
    o->bits = h->n_bits; o->bit_errors = h->n_bit_err; o->sym_errors = h->n_sym_err;
    o->near_threshold = h->n_near; o->ambiguous_windows = h->n_amb; o->windows = h->n_win;
    o->amb_rot = h->amb_r;
    o->raw_bit_errors = h->n_raw_err; o->slip_windows = h->n_slip;
    o->ber = h->n_bits ? (double)h->n_bit_err / (double)h->n_bits : 0.0;
    o->q_db = orx_q_db(o->ber);
}

void orx_destroy(orx *h)
{
    if (!h) return;
    free(h->rrc); free(h->prbs); free(h->chist); free(h->ehist); free(h->yhist); free(h->w);
    free(h->fd_Hr); free(h->fd_Hi); free(h->rhist); free(h->d_R); free(h->d_C);
    free(h->d_E); free(h->d_y); free(h->d_z); free(h->d_v); free(h->d_ahat);
    free(h->d_draw); free(h->d_berr); free(h->d_near); free(h->d_win);
    free(h);
}

/* =========================================================== CNN equaliser
 * Learned equaliser (the configured workload's alternative to the adaptive FIR
 * and phase search): input the 2-sps matched-filter output y as two channels
 * (real, imaginary); three valid 1-D convolutions of 32 channels, kernel 9,
 * each followed by GELU (exact erf form); at every symbol position an MLP
 * 32 -> 64 (GELU) -> 2 gives the soft symbol (I, Q) in unit-power units.
 * A segment of S symbols starting at symbol k0 reads y[2 k0 - 12, 2 k0 + 2 S + 12).
 * Loss: mean over the symbols of |out - target|^2.
 *
 * Parameter vector (in this order):
 *   W1[32][9][2] b1[32]  W2[32][9][32] b2[32]  W3[32][9][32] b3[32]
 *   M1[64][32] c1[64]    M2[2][64] c2[2]
 */
#define CNN_C 32
#define CNN_K 9
#define CNN_H 64
enum {
    CNN_OW1 = 0,
    CNN_OB1 = CNN_OW1 + CNN_C * CNN_K * 2,
    CNN_OW2 = CNN_OB1 + CNN_C,
    CNN_OB2 = CNN_OW2 + CNN_C * CNN_K * CNN_C,
    CNN_OW3 = CNN_OB2 + CNN_C,
    CNN_OB3 = CNN_OW3 + CNN_C * CNN_K * CNN_C,
    CNN_OM1 = CNN_OB3 + CNN_C,
    CNN_OC1 = CNN_OM1 + CNN_H * CNN_C,
    CNN_OM2 = CNN_OC1 + CNN_H,
    CNN_OC2 = CNN_OM2 + 2 * CNN_H,
    CNN_NP = CNN_OC2 + 2
};

int orx_cnn_nparams(void) { return CNN_NP; }

static double gelu(double u) { return 0.5 * u * (1.0 + erf(u / sqrt(2.0))); }
static double gelu_d(double u)
{
    return 0.5 * (1.0 + erf(u / sqrt(2.0))) + u * exp(-0.5 * u * u) / sqrt(2.0 * PI);
}

/* valid convolution: out[p][o] = b[o] + sum_t sum_c W[o][t][c] in[p + t][c] */
static void conv_fwd(const double *W, const double *b, const double *in, int Lin, int Cin, double *u)
{
    int Lout = Lin - CNN_K + 1;
    for (int p = 0; p < Lout; p++)
        for (int o = 0; o < CNN_C; o++) {
            double a = b[o];
            for (int t = 0; t < CNN_K; t++)
                for (int c = 0; c < Cin; c++) a += W[(o * CNN_K + t) * Cin + c] * in[(p + t) * Cin + c];
            u[p * CNN_C + o] = a;
        }
}

/* Loss and (optionally) gradient and outputs over nseg segments of S symbols.
 * x: nseg * (2S + 24) * 2 inputs, tgt: nseg * S * 2 targets. */
double orx_cnn_loss_grad(const double *prm, const double *x, const double *tgt, int nseg, int S, double *grad,
                         double *out)
{
    int L0 = 2 * S + 24, L1 = L0 - 8, L2 = L1 - 8, L3 = L2 - 8;
    double *u1 = xcalloc((size_t)L1 * CNN_C, sizeof(double)), *h1 = xcalloc((size_t)L1 * CNN_C, sizeof(double));
    double *u2 = xcalloc((size_t)L2 * CNN_C, sizeof(double)), *h2 = xcalloc((size_t)L2 * CNN_C, sizeof(double));
    double *u3 = xcalloc((size_t)L3 * CNN_C, sizeof(double)), *h3 = xcalloc((size_t)L3 * CNN_C, sizeof(double));
    double *dh1 = xcalloc((size_t)L1 * CNN_C, sizeof(double)), *dh2 = xcalloc((size_t)L2 * CNN_C, sizeof(double));
    double *dh3 = xcalloc((size_t)L3 * CNN_C, sizeof(double));
    double loss = 0.0;
    double norm = 1.0 / ((double)nseg * (double)S);
    if (grad) memset(grad, 0, sizeof(double) * CNN_NP);
    const double *W1 = prm + CNN_OW1, *B1 = prm + CNN_OB1, *W2 = prm + CNN_OW2, *B2 = prm + CNN_OB2;
    const double *W3 = prm + CNN_OW3, *B3 = prm + CNN_OB3, *M1 = prm + CNN_OM1, *C1 = prm + CNN_OC1;
    const double *M2 = prm + CNN_OM2, *C2 = prm + CNN_OC2;
    for (int sg = 0; sg < nseg; sg++) {
        const double *xs = x + (size_t)sg * L0 * 2;
        conv_fwd(W1, B1, xs, L0, 2, u1);
        for (int i = 0; i < L1 * CNN_C; i++) h1[i] = gelu(u1[i]);
        conv_fwd(W2, B2, h1, L1, CNN_C, u2);
        for (int i = 0; i < L2 * CNN_C; i++) h2[i] = gelu(u2[i]);
        conv_fwd(W3, B3, h2, L2, CNN_C, u3);
        for (int i = 0; i < L3 * CNN_C; i++) h3[i] = gelu(u3[i]);
        memset(dh3, 0, sizeof(double) * (size_t)L3 * CNN_C);
        for (int j = 0; j < S; j++) {
            const double *hv = h3 + (size_t)(2 * j) * CNN_C;
            double v[CNN_H], z[CNN_H], o[2];
            for (int m = 0; m < CNN_H; m++) {
                double a = C1[m];
                for (int c = 0; c < CNN_C; c++) a += M1[m * CNN_C + c] * hv[c];
                v[m] = a;
                z[m] = gelu(a);
            }
            for (int i = 0; i < 2; i++) {
                double a = C2[i];
                for (int m = 0; m < CNN_H; m++) a += M2[i * CNN_H + m] * z[m];
                o[i] = a;
            }
            const double *tg = tgt + ((size_t)sg * S + j) * 2;
            double e0 = o[0] - tg[0], e1 = o[1] - tg[1];
            loss += (e0 * e0 + e1 * e1) * norm;
            if (out) { out[((size_t)sg * S + j) * 2] = o[0]; out[((size_t)sg * S + j) * 2 + 1] = o[1]; }
            if (!grad) continue;
            double dout[2] = {2.0 * e0 * norm, 2.0 * e1 * norm}, dv[CNN_H];
            for (int i = 0; i < 2; i++) {
                grad[CNN_OC2 + i] += dout[i];
                for (int m = 0; m < CNN_H; m++) grad[CNN_OM2 + i * CNN_H + m] += dout[i] * z[m];
            }
            for (int m = 0; m < CNN_H; m++) {
                double dz = dout[0] * M2[m] + dout[1] * M2[CNN_H + m];
                dv[m] = dz * gelu_d(v[m]);
                grad[CNN_OC1 + m] += dv[m];
                for (int c = 0; c < CNN_C; c++) grad[CNN_OM1 + m * CNN_C + c] += dv[m] * hv[c];
            }
            for (int c = 0; c < CNN_C; c++) {
                double a = 0.0;
                for (int m = 0; m < CNN_H; m++) a += M1[m * CNN_C + c] * dv[m];
                dh3[(size_t)(2 * j) * CNN_C + c] = a;
            }
        }
        if (!grad) continue;
        /* backward through the three convolutions */
        struct { const double *W; double *dW, *db; const double *u, *in; double *dh_in; int Lin, Cin; double *dh; int Lout; } L[3] = {
            {W3, grad + CNN_OW3, grad + CNN_OB3, u3, h2, dh2, L2, CNN_C, dh3, L3},
            {W2, grad + CNN_OW2, grad + CNN_OB2, u2, h1, dh1, L1, CNN_C, dh2, L2},
            {W1, grad + CNN_OW1, grad + CNN_OB1, u1, xs, NULL, L0, 2, dh1, L1}};
        for (int l = 0; l < 3; l++) {
            int Cin = L[l].Cin;
            if (L[l].dh_in) memset(L[l].dh_in, 0, sizeof(double) * (size_t)L[l].Lin * Cin);
            for (int p = 0; p < L[l].Lout; p++)
                for (int o = 0; o < CNN_C; o++) {
                    double du = L[l].dh[p * CNN_C + o] * gelu_d(L[l].u[p * CNN_C + o]);
                    if (du == 0.0) continue;
                    L[l].db[o] += du;
                    for (int t = 0; t < CNN_K; t++)
                        for (int c = 0; c < Cin; c++) {
                            L[l].dW[(o * CNN_K + t) * Cin + c] += du * L[l].in[(p + t) * Cin + c];
                            if (L[l].dh_in) L[l].dh_in[(p + t) * Cin + c] += du * L[l].W[(o * CNN_K + t) * Cin + c];
                        }
                }
        }
    }
    free(u1); free(h1); free(u2); free(h2); free(u3); free(h3); free(dh1); free(dh2); free(dh3);
    return loss;
}
