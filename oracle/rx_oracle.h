/*
 * FP64 CPU oracle of the receiver DSP chain -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark use
 * this library.  The CUDA receiver never links, includes or calls it, and it
 * shares no header, table or helper with the CUDA receiver.
 *
 * It restates, in plain double-precision loops, the per-buffer receiver of
 * Sec. 2 ("Multi-Format Real-Time DSP in GPU"): 12-bit unpack, Kramers-Kronig
 * field reconstruction (square root and logarithm, overlap-save FFT Hilbert
 * transform, phase exponential) with frequency downshift, matched filter,
 * block-parallel adaptive FIR (CMA / LMS / DD-LMS), blind phase search,
 * decisions, Gray demapping and bit-error counting against PRBS-15.
 */
#ifndef RX_ORACLE_H
#define RX_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t format;      /* 0 PAM2, 1 PAM4, 2 PAM8, 3 KK-QPSK, 4 KK-16QAM            */
    int32_t sps;         /* ADC samples per symbol (PAM 2, KK 4)                      */
    int64_t buf_len;     /* samples per buffer                                         */
    int32_t pack_order;  /* 0 little-endian 24-bit words, 1 big-endian nibbles        */
    int32_t ols_n;       /* KK overlap-save Hilbert block length (power of two)        */
    int32_t ols_v;       /* KK overlap (even); outputs kept per block = ols_n - ols_v  */
    int32_t ds_num;      /* KK downshift = ds_num/ds_den cycles per sample            */
    int32_t ds_den;
    double  rrc_beta;    /* matched filter roll-off                                    */
    int32_t mf_span;     /* matched filter span in symbols (even)                      */
    int32_t ntaps;       /* adaptive FIR taps at 2 samples/symbol (odd)                */
    int32_t ntrain;      /* training symbols at stream start (multiple of win)         */
    int32_t ncma;        /* KK: leading training symbols adapted by CMA               */
    int32_t eq_block;    /* symbols per independent equaliser block (multiple of win)  */
    int32_t win;         /* symbols per LMS / blind-phase-search window                */
    double  mu;          /* decision-directed step                                     */
    double  mu_train;    /* PAM data-aided training step                               */
    double  mu_cma;      /* KK CMA step                                                */
    int32_t bps_b;       /* blind phase search test phases                             */
    int32_t amb_syms;    /* KK: payload symbols used to resolve the pi/2 ambiguity     */
    uint32_t prbs_seed;  /* PRBS-15 seed of the transmitted bits                       */
    int32_t eq_frozen;   /* KK payload: 0 taps adapt window by window inside a block;
                            1 every block filters with the call's start taps (block-
                            Toeplitz form) and one averaged step over the last block
                            gives the next call's taps                                */
    int32_t mf_mode;     /* filter before the equaliser: 0 time-domain matched filter
                            (mf_span); 1 static frequency-domain filter of fd_taps taps on
                            fd_n-point overlap-save blocks (hop fd_n/2): KK with bin-
                            truncation downsampling (fd_n/2-point inverse), PAM at the
                            input rate (fd_n-point inverse)                              */
    int32_t fd_n;        /* frequency-domain block length (power of two, >= 16)           */
    int32_t fd_taps;     /* frequency-domain filter taps (odd, <= fd_n/2 + 1)             */
    int32_t clk_track;   /* clock tracker across calls (frequency-domain form only): 1 on       */
    int64_t rs_step;     /* KK resampler to the transmitter's sample grid: 0 off; else the
                            ADC position of nominal sample m is (rs_phase0 + m rs_step) /
                            2^32 ADC samples (exact integer accumulator)                 */
    int64_t rs_phase0;
    int32_t diff_code;   /* KK: 1 = differentially quadrant-coded symbols: the first two bits
                            of a symbol (Gray) step the quadrant, the rest pick a rotation-
                            invariant point in it; decoded bits are quadrant differences  */
    int32_t eq_mode;     /* KK equaliser: 0 the block-window CMA / DD-LMS of ntaps taps with the
                            blind phase search; 1 the paper's short decision-directed LMS,
                            updated symbol by symbol, whose complex taps track the clock and
                            the symbol phase together (no phase search; ntaps 2..31, any parity) */
} orx_cfg;

typedef struct {
    int64_t calls, samples, symbols, bits, bit_errors, sym_errors;
    int64_t near_threshold, ambiguous_windows, windows;
    int64_t raw_bit_errors;  /* bit errors with no per-window re-synchronisation */
    int64_t slip_windows;    /* windows scored under a rotation other than the decoded one */
    int32_t amb_rot;     /* resolved pi/2 rotation, -1 before resolution */
    double  ber, q_db;
} orx_stats_t;

typedef struct orx orx;

/* building blocks, exported for the pins */
void    orx_unpack(const uint8_t *in, int64_t nsamp, int order, int32_t *codes);
void    orx_fft(double *re, double *im, int n, int inverse);
void    orx_hilbert_circ(const double *u, double *phi, int n);
void    orx_kk_circ(const double *intensity, double *e_re, double *e_im, int n);
void    orx_rrc(double beta, int sps, int span, double *taps);
void    orx_rrc_half(double beta, int sps, int half, double *taps);
void    orx_fd_response(const double *h, int ntaps, int n, double *H_re, double *H_im);
void    orx_fd_block(const double *x_re, const double *x_im, int n, const double *H_re, const double *H_im,
                     double *y_re, double *y_im);
void    orx_rs_taps(double mu, double *c);   /* the 16 interpolator taps at fraction mu */
void    orx_fd_clock(const double *x_re, const double *x_im, int n, const double *H_re, const double *H_im,
                     int sps, int w, double *c_re, double *c_im);
int     orx_clock_fit(const double *c_re, const double *c_im, const int64_t *center, int nblk, int sps,
                      double *ppm, double *delay);
void    orx_fd_block_full(const double *x_re, const double *x_im, int n, const double *H_re, const double *H_im,
                          double *y_re, double *y_im);
void    orx_prbs15(uint32_t seed, int64_t nbits, uint8_t *out);
double  orx_q_db(double ber);
void    orx_bps_metrics(const double *z_re, const double *z_im, int W, int mq, double s, int B,
                        double *metric);

/* CNN equaliser: parameter count, loss / gradient / outputs over segments */
int     orx_cnn_nparams(void);
double  orx_cnn_loss_grad(const double *prm, const double *x, const double *tgt, int nseg, int S,
                          double *grad, double *out);

/* streaming receiver */
orx    *orx_create(const orx_cfg *cfg);
int64_t orx_process(orx *h, const uint8_t *packed, uint8_t *bits_out, int64_t bits_cap);
/* end of the stream: decide the held-back symbols; returns the bits written, and
 * orx_process returns -1 afterwards */
int64_t orx_flush(orx *h, uint8_t *bits_out, int64_t bits_cap);
/* clock tracker across calls (cfg.clk_track = 1, mf_mode = 1): the running line fit;
 * returns the block count or -1 */
int64_t orx_clock_track(const orx *h, double *ppm, double *delay);
/* resampler from the next nominal sample on: position moved by nudge (2^-32 samples),
 * then step per nominal sample; 0 or -1 */
int     orx_set_rs(orx *h, int64_t step, int64_t nudge);
/* closed loop: re-time the resampler (step and position) from the tracker; 0 or -1 */
int     orx_clock_retime(orx *h, int64_t *step_out, int64_t *nudge_out);
int64_t orx_get(orx *h, int what, void *dst, int64_t cap, int64_t *start);
void    orx_set_taps(orx *h, const double *re, const double *im, int n);
/* static FD filter taps (zero-phase, index i + (n-1)/2): 0 or -1 */
int     orx_set_fd_taps(orx *h, const double *re, const double *im, int n);
void    orx_stats(orx *h, orx_stats_t *out);
void    orx_destroy(orx *h);

/* orx_get selectors (last call unless stated) */
enum {
    ORX_E = 1,       /* KK field E[n] (before carrier removal), complex, n in [e_prev, e)  */
    ORX_Y = 2,       /* matched-filter output y[m] after normalisation, complex             */
    ORX_Z = 3,       /* equaliser output z_k of every symbol processed in the call          */
    ORX_V = 4,       /* scaled soft value s*z_k*exp(-j*theta), complex                     */
    ORX_AHAT = 5,    /* final level-index pair (I, Q) of each processed symbol, int32 x2    */
    ORX_BERR = 6,    /* bit errors per processed symbol, int32, -1 when not counted          */
    ORX_WIN = 7,     /* per payload window: b*, m, best metric, second metric (4 doubles)   */
    ORX_TAPS = 8,    /* start taps for the next call, complex                               */
    ORX_SCAL = 9,    /* carrier re, carrier im, gain g, PAM mean, PAM std (5 doubles)       */
    ORX_NEAR = 10,   /* near-threshold flag per processed symbol, int32                      */
    ORX_DRAW = 11,   /* raw decision level-index pair before pi/2 rotation, int32 x2        */
    ORX_RS = 12,     /* resampled field on the transmitter's grid (complex)                  */
    ORX_CLK = 13     /* FD form: band-edge clock correlation C_b per emitted block (complex)   */
};

#ifdef __cplusplus
}
#endif
#endif
