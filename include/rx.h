/*
 * rx.h -- C ABI of the GPU receiver library (librx.so).
 *
 * The library implements the per-buffer receiver DSP of "Real-time,
 * Software-Defined, GPU-Based Receiver Field Trial" (arXiv 2010.14333), Sec. 2:
 * a continuous stream of 12-bit ADC buffers comes in, the binary data of the
 * recovered symbols goes out, and signal continuity is kept from one buffer to
 * the next (the overlap-save continuity the paper carries between processing
 * streams).  Two chains:
 *   - Kramers-Kronig coherent QPSK/16QAM: 12-bit unpack, square root and
 *     logarithm of the intensity, Hilbert transform by overlap-save FFT,
 *     field = sqrt(I) exp(j phase), frequency downshift, matched filter with
 *     4 -> 2 samples/symbol, adaptive FIR (CMA then decision-directed LMS),
 *     blind phase search, decision, Gray demap, bit-error count (Sec. 2, KK
 *     chain; Fig. 1c, 1d);
 *   - direct-detection PAM-2/4/8: unpack, DC removal and scaling, matched
 *     filter, LMS feed-forward equaliser (data-aided training then decision
 *     directed), decision, Gray demap, bit-error count (Sec. 2, PAM chain).
 * Every step runs in the library's own CUDA kernels on one GPU.
 *
 * Conventions
 *   - Every call returns an rx_status; nothing is thrown and nothing aborts.
 *   - The caller owns the input and output buffers and the CUDA stream; the
 *     library owns its device workspace and the stream state (allocated in
 *     rx_create on the device current at that time, released in rx_destroy).
 *   - rx_process only enqueues work on the given stream and never waits for
 *     the GPU.  Arguments are checked before anything is enqueued; errors found
 *     on the device (a bounded wait that ran out) are latched and reported by
 *     rx_stats in rx_stats_t.device_error.
 *   - One handle serves one stream of buffers; calls on one handle must be
 *     issued in stream order from one host thread.
 */
#ifndef RX_H
#define RX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rx_handle rx_handle;

typedef enum { RX_PAM2 = 0, RX_PAM4 = 1, RX_PAM8 = 2, RX_KK_QPSK = 3, RX_KK_16QAM = 4 } rx_format;

typedef enum {
    RX_OK = 0,
    RX_EINVAL = 1,    /* bad argument or configuration                            */
    RX_ENOMEM = 2,    /* device or host allocation failed                         */
    RX_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed             */
    RX_ESTATE = 4,    /* handle in an unusable state (after an earlier failure)   */
    RX_ETIMEOUT = 5,  /* a bounded device-side wait ran out (reported by stats)   */
    RX_EBOUNDS = 6    /* output capacity too small                                */
} rx_status;

/* Receiver configuration.  rx_default_config fills every field with the
 * defaults of the format; callers then change what they need. */
typedef struct {
    int32_t pack_order;  /* ADC word: 0 = little-endian 24-bit word (s0 = b0 | (b1&15)<<8,
                            s1 = b1>>4 | b2<<4), 1 = big-endian nibbles                    */
    int32_t ols_n;       /* KK overlap-save FFT length: 4096 or 65536                      */
    int32_t ols_v;       /* KK overlap, multiple of 64, < ols_n; each block keeps
                            ols_n - ols_v outputs with ols_v/2 samples of margin each side */
    int32_t ds_num;      /* KK downshift = ds_num / ds_den cycles per ADC sample (exact
                            integer phase); default 11/80 = 0.55 GHz at 4 GS/s             */
    int32_t ds_den;
    double  rrc_beta;    /* matched-filter root-raised-cosine roll-off                     */
    int32_t mf_span;     /* matched-filter span in symbols (even)                          */
    int32_t ntaps;       /* adaptive FIR taps at 2 samples/symbol, odd, <= 31               */
    int32_t ntrain;      /* training symbols at stream start, multiple of win              */
    int32_t ncma;        /* KK: leading training symbols adapted by CMA, multiple of win   */
    int32_t eq_block;    /* symbols per independently adapted block, multiple of win       */
    int32_t win;         /* symbols per LMS update / blind-phase-search window: 64         */
    double  mu;          /* decision-directed LMS step                                     */
    double  mu_train;    /* PAM data-aided training step                                   */
    double  mu_cma;      /* KK CMA step                                                    */
    int32_t bps_b;       /* KK blind-phase-search test phases, 1..32                       */
    int32_t amb_syms;    /* KK payload symbols that resolve the pi/2 ambiguity at stream
                            start (multiple of win); they are not counted in the BER       */
    uint32_t prbs_seed;  /* PRBS-15 seed of the transmitted bits (BER reference)           */
    int32_t debug;       /* 1: keep soft symbols and window metrics for rx_debug_copy      */
    int32_t fir_prec;    /* KK equaliser form (rx_fir_prec): RX_FIR_ADAPTIVE adapts the taps
                            window by window inside each block (default); the others
                            filter every payload block with the call's start taps and
                            take one averaged LMS step over the last block: FP32 on the
                            CUDA cores, or a block-Toeplitz GEMM on the tensor cores in
                            BF16, FP16 or FP8-E4M3 (per-block scaling) with FP32
                            accumulation.  The tensor-core forms need 2048 % eq_block == 0. */
    int32_t kk_front;    /* implementation of the 2^16-point KK front end (same arithmetic;
                            the carrier sums differ in rounding order only): 0 = three
                            four-step kernels (column DFT, row FFTs, column DFT + field),
                            1 = one thread-block-cluster kernel holding each block pair
                            in distributed shared memory.  Ignored for ols_n = 4096.      */
    int32_t eq_warps;    /* equaliser blocks (warps) per CTA: 0 = default (4), 2, 4 or 8   */
    int32_t mf_mode;     /* KK reduction to 2 samples/symbol (rx_mf_mode): RX_MF_TIME = the
                            time-domain matched filter of mf_span symbols (default);
                            RX_MF_FD = the static filter applied in the frequency domain on
                            overlap-save blocks of fd_n samples (hop fd_n/2) with an
                            fd_n/2-point inverse of the bins |k| < fd_n/4 as downsampler
                            (Sec. 2: FD equaliser on a 1024-point FFT, 512-point IFFT) */
    int32_t fd_n;        /* RX_MF_FD block length: power of two, 16 .. 1024; default 1024  */
    int32_t fd_taps;     /* RX_MF_FD filter taps (root-raised cosine, zero phase, unit
                            energy): odd, <= fd_n/2 + 1; default 203 (KK), 503 (PAM)      */
    int32_t clk_track;   /* 1: track the ADC clock across calls (needs RX_MF_FD): every
                            call's frequency-domain blocks feed one running estimate (the
                            band-edge delays unwrapped across buffers, a least-squares line
                            over all blocks since the last re-timing; rx_clock_track), which
                            rx_clock_retime can feed back into the resampler.  0 = off     */
    int64_t rs_step;     /* KK resampler to the transmitter's sample grid (the ADC runs on
                            its own clock; Sec. 2 recovers the clock phase in the DSP):
                            0 = off (default); else nominal sample m lies at ADC position
                            (rs_phase0 + m rs_step) / 2^32, an exact integer accumulator,
                            and the reconstructed field is interpolated there by a 16-tap
                            Hann-windowed sinc (taps j = -7..8 at the fraction rounded
                            down to 10 bits) before the filter.  Within 1 % of 2^32.     */
    int64_t rs_phase0;   /* accumulator value of nominal sample 0 (may be negative)        */
    int32_t cnn_bf16;    /* receiver CNN (rx_set_cnn) operands: 1 = BF16 (default), 0 =
                            FP16; FP32 accumulation, bias and GELU in the same packed type */
    int32_t diff_code;   /* KK: 1 = differentially quadrant-coded symbols (the transmitter
                            steps the quadrant by the Gray-decoded first two bits of a
                            symbol and picks a rotation-invariant point in it with the
                            rest): the output bits are decoded from quadrant differences, so
                            a pi/2 cycle slip costs one symbol instead of the rest of the
                            stream, and the BER counts the decoded bits against the PRBS
                            (bit_errors = raw_bit_errors).  0 = plain Gray mapping       */
    double  deadline_ms; /* per-buffer latency budget for rx_stats (Sec. 2: a buffer
                            must be processed before the stream that takes it is needed
                            again; with five streams that is five buffer durations, 5.243
                            ms for 2^22 samples at 4 GS/s).  0 = five buffer durations
                            (buf_len / fs each); > 0 = this budget in ms; < 0 = no latency
                            record (the kernels then take no timestamps)                   */
    int32_t eq_mode;     /* KK equaliser (rx_eq_mode): RX_EQ_WINDOW (default) = the adaptive
                            FIR of ntaps taps updated once per 64-symbol window, with the
                            32-phase blind phase search; RX_EQ_DD_SYMBOL = the paper's short
                            decision-directed LMS (Sec. 2, KK chain: 4 taps recover the clock
                            and symbol phase), updated after every symbol, no phase search
                            (ntaps 2..8, any parity; CMA for the first ncma training symbols).
                            Its blocks restart from the call's start taps, so it suits links
                            whose carrier phase holds still over a call (the self-coherent KK
                            link); relative laser phase noise needs the phase search          */
    int32_t pad_eq;
} rx_config;

/* Equaliser forms of the KK chain (rx_config.eq_mode). */
typedef enum { RX_EQ_WINDOW = 0, RX_EQ_DD_SYMBOL = 1 } rx_eq_mode;

/* Reduction to 2 samples/symbol of the KK chain (rx_config.mf_mode). */
typedef enum { RX_MF_TIME = 0, RX_MF_FD = 1 } rx_mf_mode;

/* Equaliser forms and precisions (rx_config.fir_prec). */
typedef enum {
    RX_FIR_ADAPTIVE = 0,
    RX_FIR_FROZEN_F32 = 1,
    RX_FIR_BF16 = 2,
    RX_FIR_FP16 = 3,
    RX_FIR_FP8 = 4
} rx_fir_prec;

typedef struct {
    int64_t calls;             /* rx_process calls                                       */
    int64_t samples;           /* ADC samples consumed                                    */
    int64_t symbols;           /* payload symbols scored                                  */
    int64_t bits;              /* payload bits scored                                     */
    int64_t bit_errors;        /* bit errors, each window scored under its best pi/2
                                  rotation (BER-tester re-synchronisation after a slip)  */
    int64_t raw_bit_errors;    /* bit errors of the decoded output with no re-sync       */
    int64_t sym_errors;        /* symbols with at least one bit error                    */
    int64_t slip_windows;      /* windows scored under a rotation other than the decoded  */
    int64_t near_threshold;    /* scored symbols whose soft value lies within 1e-4 of a
                                  decision threshold (level units)                        */
    int64_t ambiguous_windows; /* phase-search windows whose two best metrics differ by
                                  at most 1e-6 relative                                   */
    int64_t windows;           /* payload windows processed                               */
    int32_t amb_rot;           /* resolved stream-start pi/2 rotation, -1 before          */
    int32_t device_error;      /* 0, or RX_ETIMEOUT if a device-side wait ran out         */
    double  ber;               /* bit_errors / bits                                       */
    double  q_db;              /* 20 log10(sqrt(2) erfcinv(2 BER)), Sec. 3 Q-factor       */
    /* Per-buffer latency (cfg.deadline_ms >= 0): device time from the start of a
     * call's first kernel to the end of its demap (its bits in device memory),
     * read from the GPU's global timer by those kernels themselves, so that a
     * recorded call costs no API call.  The host<->device copies of the
     * host-buffer entry points are not included.  Calls inside a group round,
     * flush calls and calls that emit less than one equaliser block are not
     * recorded.  Percentiles come from a histogram of 0.5 us bins up to
     * 32.768 ms (a latency above that counts in the top bin; a percentile is
     * its bin's centre, capped at the exact maximum). */
    int64_t lat_calls;         /* calls whose latency was recorded                       */
    int64_t deadline_misses;   /* recorded calls whose latency exceeded deadline_ms      */
    double  deadline_ms;       /* the budget in force (0 when no record is kept)         */
    double  lat_p50_ms;        /* median latency (centre of its 0.5 us bin)               */
    double  lat_p99_ms;        /* 99th percentile                                         */
    double  lat_max_ms;        /* largest recorded latency (exact)                        */
} rx_stats_t;

/* Debug selectors for rx_debug_copy (each refers to the last rx_process call). */
enum {
    RX_DBG_FIELD = 1,    /* KK field E[n] before carrier removal, float2 per ADC sample     */
    RX_DBG_MF = 2,       /* matched-filter output at 2 samples/symbol: float2 (KK), float
                            (PAM)                                                           */
    RX_DBG_SOFT = 3,     /* equaliser output z_k per processed symbol, float2 (debug=1)      */
    RX_DBG_DEC = 4,      /* decision byte per payload symbol: bits 0-2 I level index,
                            bits 3-5 Q level index (before the pi/2 rotation), bit 6 near   */
    RX_DBG_WIN = 5,      /* per payload window: float4 (b*, m, best metric, second metric);
                            the metrics need debug=1                                         */
    RX_DBG_TAPS = 6,     /* start taps of the next call, float2 per tap                      */
    RX_DBG_SCAL = 7,     /* double[5]: carrier re, carrier im, gain, PAM mean, PAM 1/std     */
    RX_DBG_CODES = 8,    /* uint16 12-bit code per ADC sample of the last buffer             */
    RX_DBG_RS = 9,       /* KK field resampled to the transmitter's grid, float2 (rs_step)    */
    RX_DBG_CLK = 10      /* FD form: band-edge clock correlation per emitted block, float2   */
};

/* Defaults of a format (the workload settings of the synthetic configurations). */
rx_status rx_default_config(rx_format format, rx_config *out);

/* Create a receiver for one stream of buffers of buf_len ADC samples taken at
 * fs samples/s of a signal at baud symbols/s.  fs/baud must be 2 (PAM) or 4
 * (KK).  buf_len must be a positive multiple of 32, at most 2^30; for KK a buffer
 * may span at most about 131000 overlap-save hops (buf_len / (ols_n - ols_v)), which
 * the defaults (65536 / 4096) allow for every buf_len up to 2^30.  RX_EINVAL
 * otherwise, before any CUDA call.  cfg may be NULL (defaults).
 * Allocates all device memory up front (cudaMalloc on the current device) and
 * builds the constant tables; no kernel runs.  On success *out owns the handle. */
rx_status rx_create(rx_format format, double baud, double fs, int64_t buf_len,
                    const rx_config *cfg, rx_handle **out);

/* Process the next buffer of the stream.
 *   packed12_in: DEVICE pointer, buf_len*3/2 bytes, 16-byte aligned, packed 12-bit
 *                samples (two per three bytes, cfg.pack_order).
 *   bits_out:    DEVICE pointer with room for rx_max_bits(h)/8 bytes; receives the
 *                payload bits decided in this call, MSB first within each symbol and
 *                packed MSB first into bytes.
 *   cuda_stream: cudaStream_t (NULL = legacy default stream).
 *   nbits_out:   HOST pointer, receives the number of bits written.  The count is
 *                computed on the host from the stream position; no synchronisation.
 * Every stage emits what its full filter support allows, so outputs lag the input
 * by a fixed latency; symbols are emitted in whole equaliser blocks. */
rx_status rx_process(rx_handle *h, const uint8_t *packed12_in, uint8_t *bits_out,
                     void *cuda_stream, int64_t *nbits_out);

/* Process n consecutive buffers of the stream (ins[i], outs[i] as in rx_process;
 * nbits_out[i] per buffer).  The results are those of n rx_process calls.  The
 * stages of consecutive buffers overlap on streams the handle owns, as the paper
 * overlaps consecutive buffers in parallel streams chained by events (Sec. 2):
 * the KK field of even and odd buffers on two streams, each
 * ordered after the previous buffer's history copy and field, the matched
 * filter, the equaliser and the decisions and bits each on a stream of its own.  The pipeline starts after the work already on cuda_stream,
 * and cuda_stream waits for its last back end before anything enqueued later.
 * With cfg.debug = 1 the buffers run one at a time on cuda_stream.  The stages
 * overlap only if their streams reach separate hardware queues: with several
 * handles or groups in one process, set CUDA_DEVICE_MAX_CONNECTIONS (e.g. 32)
 * before the process first uses CUDA. */
rx_status rx_process_batch(rx_handle *h, const uint8_t *const *ins, uint8_t *const *outs, int n,
                           void *cuda_stream, int64_t *nbits_out);

/* Same as rx_process with HOST buffers: copies the input host->device, runs the
 * chain and copies the bits device->host, all enqueued on cuda_stream.  For
 * asynchronous copies the host buffers must be page-locked.  Returns after
 * enqueuing; the bits are valid once the stream has reached this point. */
rx_status rx_process_host(rx_handle *h, const uint8_t *host_in, uint8_t *host_bits_out,
                          void *cuda_stream, int64_t *nbits_out);

/* rx_process_batch with HOST buffers (page-locked for the copies to overlap):
 * host_ins[i] holds buffer i as packed 12-bit bytes, host_outs[i] receives its
 * bits (capacity rx_max_bits / 8 + 1 bytes).  The copies to the device run on a
 * stream the handle owns, into four device staging slots, so the copy of buffer
 * i+1 (up to i+3) overlaps the front end of buffer i; each buffer's bits are
 * copied back after its demap.  The outputs are valid once cuda_stream has
 * reached the end of the call. */
rx_status rx_process_host_batch(rx_handle *h, const uint8_t *const *host_ins, uint8_t *const *host_outs, int n,
                                void *cuda_stream, int64_t *nbits_out);

/* Upper bound of the bits one rx_process or rx_flush call can emit. */
int64_t rx_max_bits(const rx_handle *h);

/* End of the stream: emit the payload symbols the last buffers still hold back.
 * Every stage of the chain lags the input (the KK overlap-save margin, the filter
 * and equaliser supports, whole equaliser blocks), so after the last rx_process
 * the symbols of the stream's final few thousand samples have not been decided.
 * rx_flush pads the stream after its last sample with that sample's code
 * repeated (the mirror of the stream start, where the first sample is
 * replicated) and runs the chain until every symbol whose centre lies inside the
 * stream has been decided.  The pad buffers reuse the per-call carrier and gain
 * (KK) or mean and standard deviation (PAM) of the last real buffer.
 *   bits_out:  DEVICE pointer with room for rx_max_bits(h)/8 bytes; receives the
 *              bits of payload symbols [first undecided, last in the stream].
 *   nbits_out: HOST pointer, the number of bits written (computed on the host).
 * Windows whose last symbol lies within ceil((mf_span + ntaps) / 2) symbols of
 * the stream end are decided but not scored in rx_stats (their filter supports
 * reach into the pad).  Enqueued on cuda_stream, which must be the stream (or
 * follow the stream) of the last rx_process call.  After rx_flush the handle
 * accepts no more buffers (RX_ESTATE); a second rx_flush emits nothing. */
rx_status rx_flush(rx_handle *h, uint8_t *bits_out, void *cuda_stream, int64_t *nbits_out);

/* Resampler accumulator for a measured ADC clock (rx_clock_estimate's result):
 * ADC sample n lies at transmitter time delay + n (1 + 1e-6 ppm) nominal samples
 * (Sec. 2: the ADC runs on its own clock and the DSP recovers the clock phase).
 * The resampler reads nominal sample m at ADC position (rs_phase0 + m rs_step) /
 * 2^32 = (m - delay) / (1 + 1e-6 ppm).  With the ADC period P = round((1 + 1e-6
 * ppm) 2^32) and the delay D = round(delay 2^32), both in units of 2^-32 samples
 * and rounded to nearest (ties to even) from the double product:
 * rs_step = floor((2^64 + floor(P/2)) / P) and rs_phase0 = -floor((D 2^32 +
 * floor(P/2)) / P), in exact 128-bit integer arithmetic.  RX_EINVAL unless
 * |ppm| < 9000 and |delay| < 2^30 (rx_create accepts rs_step within 1 % of 2^32). */
rx_status rx_resampler_from_clock(double ppm, double delay, int64_t *rs_step, int64_t *rs_phase0);

/* Taps of the static frequency-domain filter (mf_mode = RX_MF_FD), in place of
 * the root-raised-cosine taps it starts with (Sec. 2: both chains filter with a
 * static frequency-domain equaliser whose taps come from the link; the paper does
 * not publish them).  re / im: HOST arrays of n taps h_i, i = -(n-1)/2 .. (n-1)/2
 * in that order (index 0 holds h_{-(n-1)/2}); im may be NULL (real taps) and must
 * be NULL or all zero for PAM, whose filter output is taken as real.  n odd,
 * 1 <= n <= fd_n / 2 + 1.  The filter's response at the kept bins is recomputed
 * on the host and copied after the device has finished all work (synchronous);
 * calls made afterwards use it.  RX_EINVAL for other arguments or a handle
 * without the frequency-domain form. */
rx_status rx_set_fd_taps(rx_handle *h, const double *re, const double *im, int n);

/* Least-squares fit of static filter taps to a training capture (the calibration
 * that gives rx_set_fd_taps its taps):
 *   minimise  sum_{k=0}^{na-1} | a_k - sum_{i=-L}^{L} h_i x[first + step k - i] |^2
 *             + ridge (trace(R) / n) sum_i |h_i|^2
 * over n = ntaps = 2L + 1 taps, R the normal matrix X^H X of the data matrix
 * X[k][i] = x[first + step k - i].  x: HOST, nx samples at the filter's input rate
 * (x_im NULL for real data); a: HOST, na targets (a_im NULL for real targets);
 * step: input samples per target (PAM 2, KK 4 for one target per symbol).  The
 * normal equations are formed in FP64 (the first `step` rows of R directly, the
 * rest by the shift recurrence R[i+step][j+step] = R[i][j] + the term of the
 * target before the first minus that of the last) and solved by Cholesky
 * factorisation.  Output h_re / h_im (n values, ordered as rx_set_fd_taps takes
 * them); h_im may be NULL only for real data and targets (then the taps are
 * real).  RX_EINVAL unless ntaps is odd in [1, 2049], step >= 1, na >= ntaps,
 * first >= L and first + step (na - 1) + L < nx, or when R + ridge is not
 * positive definite.  Host only; no device is used. */
rx_status rx_fd_ls_taps(const double *x_re, const double *x_im, int64_t nx, int64_t first, int step,
                        const double *a_re, const double *a_im, int64_t na, int ntaps, double ridge,
                        double *h_re, double *h_im);

/* Synchronises cuda_stream, then copies the accumulated counters. */
rx_status rx_stats(rx_handle *h, rx_stats_t *out, void *cuda_stream);

/* Copies an intermediate of the last call to HOST memory dst (capacity cap
 * elements of the selector's type) after synchronising cuda_stream.  *count
 * receives the number of elements available and *start the stream index of the
 * first one (ADC sample, 2-sps sample, symbol or window, as the selector says). */
rx_status rx_debug_copy(rx_handle *h, int what, void *dst, int64_t cap, int64_t *count,
                        int64_t *start, void *cuda_stream);

/* Replace the taps the next call starts from (HOST arrays of n <= ntaps values;
 * im may be NULL for PAM).  Synchronous. */
rx_status rx_set_taps(rx_handle *h, const double *re, const double *im, int n);

/* Stage timing.  rx_profile(h, n) with n >= 1 makes every n-th later call
 * (those whose call index is a multiple of n) record a CUDA event before and
 * after each stage, on the stream that runs the stage (unpack, K1a forward
 * radix-16, K1b row FFTs, K1c field assembly, matched filter, equaliser,
 * demap); rx_profile(h, 0) stops.  Sampling keeps the cost of the events off
 * most calls of a long run.  rx_profile_read waits for the recorded
 * calls, writes the summed milliseconds of each stage to ms[0..n-1] (n <= 7,
 * in the order above; a stage a format lacks reads 0) and the number of calls
 * measured to *calls, and clears the record. */
rx_status rx_profile(rx_handle *h, int enable);
rx_status rx_profile_read(rx_handle *h, double *ms, int n, int64_t *calls);

/* Block-Toeplitz FIR with fixed taps on the tensor cores: the equaliser's
 * filter in its frozen form (Sec. 2 equaliser; precision forms of the FIR
 * contraction), exposed on its own so that its rounding can be measured.
 *   z[k] = sum_{i=0}^{ntaps-1} conj(w[i]) y[2k + ntaps - 1 - i],  k = 0 .. nsym-1
 * y:      DEVICE, complex FP32 interleaved (re, im), ny samples at 2 samples per
 *         symbol, 16-byte aligned; ny >= 2 nsym + ntaps + 1.
 * w:      DEVICE, ntaps complex FP32 taps (odd ntaps <= 31).
 * prec:   RX_FIR_BF16, RX_FIR_FP16 or RX_FIR_FP8 (operands rounded to that type,
 *         FP32 accumulation; FP8 scales y by a power of two per block of
 *         scale_block symbols and w by one power of two, both undone on output).
 * nsym:   multiple of 16; scale_block: multiple of 16 dividing 2048 and nsym.
 * z_out:  DEVICE, nsym complex FP32, 16-byte aligned.
 * status: DEVICE int32 the caller zeroed; a device-side wait that ran out writes
 *         RX_ETIMEOUT there.
 * Enqueued on cuda_stream; returns RX_EINVAL for bad arguments before launching. */
rx_status rx_fir_block(const float *y, int64_t ny, const float *w, int ntaps, int prec, int64_t nsym,
                       int scale_block, float *z_out, int32_t *status, void *cuda_stream);

/* Groups: many independent streams per submission (the paper's receiver runs
 * one stream per format; a group serves many at once, of any formats and buffer
 * lengths).  A group holds n existing handles (not owned; each must be used
 * only through the group while it exists) and processes one buffer of every
 * member per rx_group_process call: ins[i], outs[i] and nbits_out[i] as in
 * rx_process for member i.  Results equal those of n rx_process calls.
 * Members run concurrently on up to 8 worker streams the group owns, forked
 * from cuda_stream and joined back into it.
 *   RX_GROUP_GRAPH: each round is captured into a CUDA graph, the executable
 *     graph is updated in place and launched once (cuda_stream must not be the
 *     legacy default stream).  A failed capture leaves the members in RX_ESTATE.
 *   RX_GROUP_TUNE:  at creation, each distinct member shape (format, buffer
 *     length, configuration) times its implementation choices on pseudo-random
 *     input and keeps the fastest: the 2^16-point front-end structure
 *     (kk_front 0 / 1) and the equaliser CTA shape (eq_warps 2 / 4 / 8).  The
 *     choice of eq_warps leaves every output bit-identical; kk_front changes
 *     only the summation order of the carrier estimate.  rx_group_tuning reports
 *     the choice for member i. */
typedef struct rx_group rx_group;
enum { RX_GROUP_GRAPH = 1, RX_GROUP_TUNE = 2 };
rx_status rx_group_create(rx_handle *const *members, int n, int flags, rx_group **out);
rx_status rx_group_process(rx_group *g, const uint8_t *const *ins, uint8_t *const *outs, void *cuda_stream,
                           int64_t *nbits_out);
rx_status rx_group_tuning(const rx_group *g, int i, int32_t *kk_front, int32_t *eq_warps);
rx_status rx_group_destroy(rx_group *g);

/* Kramers-Kronig field of one buffer without any device allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory once they are running.  Examples are a real-time
 * ingest thread that must not stall on cudaMalloc (which can synchronise the
 * device), code running inside another framework whose device memory belongs
 * to that framework's allocator, and plugin hosts that forbid allocations after
 * start-up.  It computes what rx_process emits as RX_DBG_FIELD for the first
 * buffer of a stream: 12-bit unpack, overlap-save Hilbert transform of
 * ln(I)/2 and E = sqrt(I) exp(j phi), for stream samples [0, nsamp - ols_v/2).
 *
 *   packed12_in: DEVICE pointer, nsamp*3/2 bytes, 16-byte aligned.
 *   nsamp:       multiple of 32, at most 524288 (2^19) samples, and the overlap-save
 *                blocks must fit the FFT rows: ceil(J/2) * ols_n <= 2^19 complex
 *                values with J = ceil((nsamp - ols_v/2) / (ols_n - ols_v)) blocks
 *                (at ols_n = 65536 and nsamp = 2^19 that allows ols_v up to 4096).
 *   ols_n/ols_v: as in rx_config (4096 or 65536; overlap a multiple of 64, < ols_n).
 *   field_out:   DEVICE pointer, 8-byte aligned, room for 2*(nsamp - ols_v/2)
 *                floats (interleaved real, imaginary).
 *
 * The scratch (twiddle and ln tables, a packed-history region, FFT rows, field,
 * carrier sums) is one fixed device array of about 8.1 MiB in librx.so;
 * every GPU that loads the library holds it until the process exits.  Sizes
 * beyond the limits return RX_EINVAL before anything is enqueued.  The call
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine); it
 * enqueues its kernels on cuda_stream and returns.  The first call on a device
 * does a one-time set-up with that device current: it looks up the array's
 * device address and copies the tables on cuda_stream, then synchronises that
 * stream, so make that first call before any stream capture.  Host threads that
 * make their first calls at the same time do the set-up once (it is serialised).
 * All calls share the one array and it keeps the last call's contents, so calls
 * that overlap on the GPU (on different streams or from different threads) race
 * and corrupt each other's results; issue them in order on one stream.  Returns
 * RX_ECUDA when the set-up or a launch fails. */
rx_status rx_kk_field_noalloc(const uint8_t *packed12_in, int64_t nsamp, int32_t pack_order,
                              int32_t ols_n, int32_t ols_v, float *field_out, void *cuda_stream);

/* ------------------------------------------------------------------ CNN
 * Learned equaliser (the configured workload's alternative to the adaptive FIR
 * and blind phase search, trained on the GPU by the library's own kernels).
 * Input: the 2-sps matched-filter output y (complex, as RX_DBG_MF).  Three valid
 * convolutions of 32 channels, kernel 9, each followed by GELU (exact erf); at
 * every symbol position an MLP 32 -> 64 (GELU) -> 2 gives the soft symbol in
 * unit-power units.  A segment of 64 symbols starting at symbol k0 reads
 * y[2 k0 - 12, 2 k0 + 140).  Parameters (rx_cnn_nparams() floats, in order):
 *   W1[32][9][2] b1[32] W2[32][9][32] b2[32] W3[32][9][32] b3[32]
 *   M1[64][32] c1[64] M2[2][64] c2[2].
 * The forward convolutions run on the tensor cores with BF16 operands and FP32
 * accumulation; gradients and Adam (beta 0.9 / 0.999, eps 1e-8) are FP32 on FP32
 * master weights.  Loss: mean over symbols of |out - target|^2. */
typedef struct rx_cnn rx_cnn;

int       rx_cnn_nparams(void);
/* Allocates parameters, Adam state and activation storage for up to max_seg
 * segments per gradient call (device memory on the current device). */
rx_status rx_cnn_create(int max_seg, rx_cnn **out);
/* HOST float arrays of rx_cnn_nparams() values; set resets the Adam state.
 * Both synchronise the device. */
rx_status rx_cnn_set_params(rx_cnn *c, const float *params, int n);
rx_status rx_cnn_get_params(rx_cnn *c, float *params, int n);
/* DEVICE pointers: y complex float pairs; seg_start[s] = index in y of segment
 * s's first input sample (2 k0 - 12); out receives nseg * 64 * 2 floats. */
rx_status rx_cnn_forward(rx_cnn *c, const float *y, const int64_t *seg_start, int nseg, float *out,
                         void *cuda_stream);
/* Gradient of the loss over nseg <= max_seg segments with DEVICE targets
 * tgt[nseg][64][2]; grad_out (DEVICE, rx_cnn_nparams() floats) and loss_out
 * (DEVICE, one float) may be NULL.  The gradient is kept for rx_cnn_adam_step. */
rx_status rx_cnn_grad(rx_cnn *c, const float *y, const int64_t *seg_start, const float *tgt, int nseg,
                      float *grad_out, float *loss_out, void *cuda_stream);
rx_status rx_cnn_adam_step(rx_cnn *c, float lr, void *cuda_stream);
void      rx_cnn_destroy(rx_cnn *c);

/* Use the CNN (NULL: back to the adaptive FIR) for the payload decisions of a KK
 * receiver from its next call on.  The network is borrowed: keep it alive while
 * the receiver uses it. */
rx_status rx_set_cnn(rx_handle *h, const rx_cnn *cnn);

/* Releases the device memory and the handle.  NULL is ignored. */
void rx_destroy(rx_handle *h);

/* Static description of a status code. */
const char *rx_strerror(rx_status s);

/* ADC clock estimate from the last call (mf_mode = RX_MF_FD, KK or PAM chain; Sec. 2
 * recovers the clock phase in the frequency domain block by block, in the PAM chain
 * after its static FD filter).  With P the samples per symbol (4 KK, 2 PAM) and
 * S = N / P the bin of the symbol rate, each frequency-domain block b correlates its
 * filtered spectrum at +1/(2T) with its image one symbol rate lower,
 * C_b = sum_{|k - S/2| <= w} Y_k conj(Y_{k - S}) (w the roll-off half-width
 * ceil(beta S / 2) in bins, at most 31); a symbol grid at ADC positions d (mod P)
 * gives arg C_b = -2 pi d / P.  The unwrapped d_b over the call's blocks are fitted
 * by the line d_b = -delay - 1e-6 ppm centre_b: *ppm is the ADC clock offset (sample
 * period (1 + 1e-6 ppm) nominal samples), *delay the transmitter time of ADC sample 0
 * in samples, in (-P/2, P/2] (the whole-symbol ambiguity is not resolved).  With the
 * KK resampler on, the estimate is the residual against its accumulator.
 * Synchronises the stream.  RX_EINVAL without the FD form, RX_ESTATE with fewer
 * than 2 blocks. */
rx_status rx_clock_estimate(rx_handle *h, double *ppm, double *delay, void *cuda_stream);

/* Running ADC clock estimate (rx_config.clk_track = 1): the band-edge delays of every
 * call's frequency-domain blocks (as in rx_clock_estimate), unwrapped across buffers
 * (the first block of a call against the last of the previous one; Sec. 2 unwraps the
 * clock phase with the previous buffer's stream), fitted by one least-squares line
 * over all blocks since the stream start or the last re-timing.  *ppm, *delay as in
 * rx_clock_estimate (with the resampler on: the residual against its accumulator);
 * *nblocks the blocks fitted.  Synchronises the stream.  RX_EINVAL without
 * clk_track, RX_ESTATE with fewer than 2 blocks. */
rx_status rx_clock_track(rx_handle *h, double *ppm, double *delay, int64_t *nblocks, void *cuda_stream);

/* Closed clock loop, run between calls (KK chain with the resampler and clk_track):
 * the running fit y(c) = y0 + s c of the unwrapped block delays (the symbol grid sits
 * at resampled positions congruent to y mod 4) re-times the resampler from the next
 * nominal sample r on: the step becomes round(step (1 + s)) and the accumulator at r
 * moves by round(w step), w = y(r) wrapped into (-2, 2] (whole symbols are not
 * observable and are left alone); halves round away from zero.  The tracker then
 * restarts.  *step_out / *nudge_out (nullable) receive the applied values.
 * Synchronises the stream.  RX_EINVAL without the resampler or clk_track, RX_ESTATE
 * with fewer than 2 blocks, RX_EBOUNDS when the step would leave 1 % of 2^32. */
rx_status rx_clock_retime(rx_handle *h, int64_t *step_out, int64_t *nudge_out, void *cuda_stream);

/* Re-time the resampler by hand from the next nominal sample on: its accumulator
 * moves by nudge (units of 2^-32 ADC samples, |nudge| < 2^36) and then advances by
 * step per nominal sample (within 1 % of 2^32).  The clock tracker restarts.
 * Synchronises the stream.  RX_EINVAL without the resampler or out of range. */
rx_status rx_set_resampler(rx_handle *h, int64_t step, int64_t nudge, void *cuda_stream);

/* Self-test of the bounded device waits: one CTA waits for an mbarrier phase that
 * nothing completes, gives up after a bounded number of polls (as every wait of the
 * receiver kernels does) and reports it.  Returns RX_ETIMEOUT when the bound worked
 * (the expected result), RX_OK if the phase somehow completed, RX_ECUDA on a CUDA
 * error.  Synchronises the stream; the context stays usable. */
rx_status rx_selftest_wait_timeout(void *cuda_stream);

/* FP32 arithmetic rate of this GPU, measured: every SM runs resident CTAs whose threads
 * each advance 8 independent FMA chains for `iters` steps (16 iters flop per thread),
 * timed with CUDA events on the stream (after one untimed launch).  *tflops receives
 * flop / time in TFLOP/s, the denominator of the ALU rooflines measured on the part as
 * it runs (clock and power as they are); the values the chains end with go to a
 * device word so that no FMA is removed.  iters in [1, 2^24].  Synchronises the
 * stream.  Not part of the receiver: the paper has no counterpart. */
rx_status rx_selftest_fma_rate(int iters, double *tflops, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* RX_H */
