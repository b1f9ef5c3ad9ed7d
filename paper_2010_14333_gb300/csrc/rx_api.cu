// C ABI of the receiver library: handle lifetime, per-call scheduling of the
// kernels, constant tables, statistics and debug copies.  See include/rx.h.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <cmath>
#include <complex>
#include <vector>

#include <cuda_runtime.h>

#include "rx_async.cuh"
#include "rx_internal.cuh"

using namespace rxk;

// RX_TRACE=1 in the environment: report each failing CUDA call of the library on
// stderr (name and place), for diagnosing a status of RX_ECUDA
static bool trace_on()
{
    static int on = -1;
    if (on < 0) {
        const char *v = getenv("RX_TRACE");
        on = (v && *v && *v != '0') ? 1 : 0;
    }
    return on == 1;
}
static cudaError_t traced(cudaError_t e, const char *where)
{
    if (e != cudaSuccess && trace_on()) fprintf(stderr, "rx: %s failed: %s\n", where, cudaGetErrorName(e));
    return e;
}

struct rx_handle {
    int fmt, kk, bps, mq, sps, decim, hmf, th;
    long long nb;
    rx_config cfg;
    EqParams ep;
    int nhist;                      // codes kept before a buffer
    int N, V, hop, N2;              // KK overlap-save geometry
    int npairs_max;
    // stream position (host mirror of the deterministic schedule)
    long long calls, e_prev, f_prev, q_prev;
    int trained, amb_done;
    int cw, ew, yw, tw, uw;         // ping-pong indices
    long long ebase_cur, ybase_cur; // stream index of element 0 of E[ew], Y[yw]
    // last call, for rx_debug_copy
    long long l_e_prev, l_e_k, l_f_prev, l_f_k, l_sym_lo, l_pay_lo, l_q_k;
    int l_nwin;
    int broken;
    // device memory
    uint16_t *codes[2];
    uint8_t *phist[3];              // KK: packed history, three slots (see front2)
    int hw;
    float2 *fftws[2], *E[kSlots];   // FFT workspace per front-end stream
    void *Y[kSlots];
    uint8_t *dec[kSlots], *winb[kSlots], *prbs;
    uint32_t *prbs_bits;            // the PRBS period bit-packed MSB first, first 256 bits repeated
    uint4 *winrec[kSlots];          // per payload window: errors under the four rotations, near count
    int l_ds;                       // decision slot of the last call
    // pipeline of rx_process_batch: the front end (field, matched filter) of
    // buffer i+1 runs while the back end (equaliser, demap) of buffer i runs on
    // `back` / `tail`
    // KK: the field of odd calls runs on `front2`, so that the field of call i+1
    // overlaps the field of call i; its forward pass waits only for the history
    // copy of call i (ev_hist) and its inverse pass for the field of call i
    // (ev_front).  Call i+1 writes the history slot that call i-1 read, hence
    // three slots.
    cudaStream_t front, front2, mid, back, tail, copy;   // KK: field | matched filter | equaliser | demap
    cudaEvent_t ev_fork, ev_front, ev_hist, ev_join, ev_yfree[kSlots], ev_efree[kSlots],
        ev_dfree[kSlots], ev_inready[kInSlots], ev_infree[kInSlots], ev_cfree[2];
    float2 *taps[2], *twN, *twN2, *ds_tab;
    float *lnt;
    float *rrc;
    float rrc_host[2 * 64 + 1];     // host copy of the matched-filter taps
    float4 *dbg_win;
    float2 *dbg_z;
    DevState *st;
    uint8_t *in_stage[kInSlots], *bits_stage;   // device staging of the host-buffer entry points
    float2 *zbuf;                   // payload soft symbols of the tensor-core FIR forms
    float2 *gpart;                  // frozen forms: tap-gradient partials, one row of 32 per window
    int rs;                         // resampler of the KK field to the transmitter's grid
    float2 *R[2];                   // resampled field ping-pong [kEHist history | call]
    int rw;                         // R slot of the last call
    long long r_prev, rbase_cur, l_r_prev, l_r_k;
    float *rs_tab;                  // 1024 x 16 interpolator taps
    int fd;                         // frequency-domain reduction to 2 samples/symbol
    float2 *fd_H, *fd_tw;           // its kept-bin response (times 1/N) and N-point twiddles
    float2 *clk;                    // KK FD: band-edge clock correlation of each block of the last call
    int clk_w;                      // its half-width in bins
    long long dec_cap, win_cap, y_cap;
    int nsm;                        // SMs of the handle's device
    // stage timing: a ring of event sets, one per profiled call
    const rx_cnn *cnn;              // learned equaliser for the payload, or null
    int prof_on;               // sampling period in calls (0: off)
    int prof_cur;              // the call being enqueued is sampled
    cudaEvent_t *prof_ev;      // kProfRing * 2 * kStages events (begin, end of every stage)
    int *prof_used;            // stages recorded in each ring slot (bitmask)
    long long prof_head, prof_tail;
    double prof_ms[8];
    long long prof_calls;
    // per-buffer latency record, kept on the device clock by the call's first kernel
    // and its demap (no API call per buffer)
    double lat_budget;         // ms; 0 = no record
    LatRecord *lat_dev;        // device record, or null
    long long lat_head;        // recorded calls enqueued (slot = lat_head % kLatSlots)
    uint32_t *lat_hist;        // host copy of the histogram for rx_stats
    int in_group;              // the call is part of a group round (not recorded)
    // end of stream (rx_flush)
    int flushed;               // rx_flush ran: no more buffers
    int flush_mode;            // the call being enqueued is a pad call of rx_flush
    int flush_par;             // PAM: sums slot (call index mod 3) of the last real call (its mean and deviation)
    long long flush_score_end; // windows reaching this symbol are not scored
    long long flush_bits;      // bound of the bits rx_flush emits
    long long pad_calls;       // pad calls run by rx_flush (not counted as input)
    // resampler accumulator, piecewise: nominal sample m >= rs_r0 lies at ADC position
    // (rs_psi0 + (m - rs_r0) cfg.rs_step) / 2^32 (a re-timing starts a new piece)
    long long rs_r0;
    __int128 rs_psi0;
};

static const double kLatBinMs = (double)kLatBinNs * 1e-6;

// percentile p of n recorded latencies (centre of its bin), 0 without records
static double lat_pct(const uint32_t *hist, long long n, double max_ms, double p)
{
    if (n <= 0) return 0.0;
    long long want = (long long)ceil(p * (double)n), acc = 0;
    if (want < 1) want = 1;
    for (int b = 0; b < kLatBins; b++) {
        acc += hist[b];
        if (acc >= want) return fmin(((double)b + 0.5) * kLatBinMs, max_ms);
    }
    return max_ms;
}

static const int kProfRing = 1024;
static const int kStages = 7;        // unpack, kk_fwd, kk_rows, kk_inv, mf, eq, demap
static const int kEvPerCall = 2 * kStages;

// begin / end event of a stage, on the stream that runs it
static void prof_begin(rx_handle *h, int stage, cudaStream_t st)
{
    if (!h->prof_cur) return;
    long long slot = h->prof_head % kProfRing;
    cudaEventRecord(h->prof_ev[slot * kEvPerCall + 2 * stage], st);
    h->prof_used[slot] |= 1 << stage;
}
static void prof_end(rx_handle *h, int stage, cudaStream_t st)
{
    if (!h->prof_cur) return;
    long long slot = h->prof_head % kProfRing;
    cudaEventRecord(h->prof_ev[slot * kEvPerCall + 2 * stage + 1], st);
}

// hook of the K1 launcher: s > 0 begins stage s; s < 0 ends stage -s-1 and, up to
// stage 3, begins stage -s
void rxk::prof_stage(void *prof, int stage, cudaStream_t st)
{
    if (!prof) return;
    rx_handle *h = (rx_handle *)prof;
    if (stage > 0) {
        prof_begin(h, stage, st);
    } else {
        prof_end(h, -stage - 1, st);
        if (-stage <= 3) prof_begin(h, -stage, st);
    }
}

// harvest the oldest recorded call (blocking on its events)
static void prof_harvest_one(rx_handle *h)
{
    long long slot = h->prof_tail % kProfRing;
    int used = h->prof_used[slot];
    cudaEvent_t *ev = h->prof_ev + slot * kEvPerCall;
    for (int s = 0; s < kStages; s++) {
        if (!(used & (1 << s))) continue;
        cudaEventSynchronize(ev[2 * s + 1]);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[2 * s], ev[2 * s + 1]) == cudaSuccess) h->prof_ms[s] += ms;
    }
    h->prof_used[slot] = 0;
    h->prof_tail++;
    h->prof_calls++;
}

// ---------------------------------------------------------------- host tables
// Root-raised cosine, sps*span+1 taps, unit energy, zero phase (textbook form).
static void rrc_half(double beta, int sps, int half, double *h);
static void rrc_taps(double beta, int sps, int span, double *h) { rrc_half(beta, sps, sps * span / 2, h); }
// the same pulse with 2 half + 1 taps
static void rrc_half(double beta, int sps, int half, double *h)
{
    const double pi = 3.14159265358979323846;
    int n = 2 * half + 1;
    double e = 0;
    for (int i = 0; i < n; i++) {
        double t = (double)(i - half) / sps, v;
        if (fabs(t) < 1e-12) {
            v = 1.0 - beta + 4.0 * beta / pi;
        } else if (beta > 0 && fabs(fabs(4.0 * beta * t) - 1.0) < 1e-12) {
            v = beta / sqrt(2.0) * ((1 + 2 / pi) * sin(pi / (4 * beta)) + (1 - 2 / pi) * cos(pi / (4 * beta)));
        } else {
            double den = pi * t * (1.0 - 16.0 * beta * beta * t * t);
            v = (sin(pi * t * (1 - beta)) + 4 * beta * t * cos(pi * t * (1 + beta))) / den;
        }
        h[i] = v;
        e += v * v;
    }
    for (int i = 0; i < n; i++) h[i] /= sqrt(e);
}

// PRBS-15 (x^15 + x^14 + 1) one period, register seeded with (seed mod 32767) + 1.
static void prbs15_period(uint32_t seed, uint8_t *out)
{
    uint32_t r = seed % 32767u + 1u;
    for (int i = 0; i < 32767; i++) {
        uint32_t b = ((r >> 13) ^ (r >> 14)) & 1u;
        r = ((r << 1) | b) & 0x7FFFu;
        out[i] = (uint8_t)b;
    }
}

static void twiddles(int n, float2 *out)   // e^{-2 pi i k / n}
{
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < n; k++) {
        double a = -2.0 * pi * (double)k / (double)n;
        out[k] = make_float2((float)cos(a), (float)sin(a));
    }
}

// ------------------------------------------------------------------- schedule
struct Sched {
    long long avail, e_k, r_k, f_k, s_k, q_k;
};
// accumulator of nominal sample m (>= rs_r0) and the count of nominal samples whose
// accumulator lies below lim (lim at or beyond the accumulator at rs_r0), exact in
// 128-bit integers
static __int128 rs_psi(const rx_handle *h, long long m)
{
    return h->rs_psi0 + (__int128)(m - h->rs_r0) * h->cfg.rs_step;
}
static long long rs_below(const rx_handle *h, __int128 lim)
{
    __int128 d = lim - h->rs_psi0;
    if (d <= 0) return h->rs_r0;
    return h->rs_r0 + (long long)((d + h->cfg.rs_step - 1) / h->cfg.rs_step);
}
// nominal samples the resampler can emit from the field [0, e_k): #{m >= 0 :
// floor(psi_m / 2^32) + 8 < e_k}
static long long rs_count(const rx_handle *h, long long e_k)
{
    return rs_below(h, (__int128)(e_k - 8) << 32);
}
static Sched schedule(const rx_handle *h, long long calls, long long q_prev)
{
    Sched s;
    s.avail = (calls + 1) * h->nb;
    s.e_k = h->kk ? s.avail - h->V / 2 : s.avail;
    if (s.e_k < 0) s.e_k = 0;
    s.r_k = h->rs ? rs_count(h, s.e_k) : s.e_k;   // the filter's input on its own grid
    if (h->rs && s.r_k < h->r_prev) s.r_k = h->r_prev;
    s.f_k = (s.r_k >= h->hmf + 1) ? (s.r_k - h->hmf - 1) / h->decim + 1 : 0;
    if (h->fd) {   // whole frequency-domain blocks: block b reads up to N/2 b + 3N/4
        long long N = h->cfg.fd_n, bk = (s.r_k >= 3 * N / 4) ? (s.r_k - 3 * N / 4) / (N / 2) + 1 : 0;
        s.f_k = bk * (N / 2) / h->decim;
    }
    s.s_k = (s.f_k >= h->th + 1) ? (s.f_k - h->th - 1) / 2 + 1 : 0;
    long long nt = h->cfg.ntrain, B = h->cfg.eq_block;
    s.q_k = (s.s_k >= nt) ? nt + ((s.s_k - nt) / B) * B : 0;
    if (s.q_k < q_prev) s.q_k = q_prev;
    return s;
}

// Pad buffer of rx_flush: the stream's last 12-bit code repeated, packed two per
// three bytes in the handle's order.  The code is read from the packed history of
// the last call (KK: its last pair) or from the last unpacked code (PAM).
__global__ void k_pad_fill(uint8_t *dst, long long nbytes, const uint8_t *hist_end, const uint16_t *code, int order)
{
    uint32_t c;
    if (hist_end) {
        uint32_t b1 = hist_end[-2], b2 = hist_end[-1];   // the pair's last two bytes
        c = order == 0 ? (b1 >> 4) | (b2 << 4) : ((b1 & 0xFu) << 8) | b2;   // second sample of the pair
    } else {
        c = *code;
    }
    uint8_t pat[3];
    if (order == 0) {   // s0 = b0 | (b1 & 15) << 8, s1 = b1 >> 4 | b2 << 4
        pat[0] = (uint8_t)(c & 0xFF);
        pat[1] = (uint8_t)((c >> 8) | ((c & 0xF) << 4));
        pat[2] = (uint8_t)(c >> 4);
    } else {            // s0 = b0 << 4 | b1 >> 4, s1 = (b1 & 15) << 8 | b2
        pat[0] = (uint8_t)(c >> 4);
        pat[1] = (uint8_t)(((c & 0xF) << 4) | (c >> 8));
        pat[2] = (uint8_t)(c & 0xFF);
    }
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nbytes; i += (long long)gridDim.x * blockDim.x)
        dst[i] = pat[i % 3];
}

// Clock tracker across calls (one CTA): the band-edge delay d_b = -(P / 2 pi) arg C_b of
// each of this call's nblk blocks (global block index b0 + i, centre (N/2) b + N/4),
// unwrapped block to block (one period P added or taken away when consecutive delays
// differ by more than P/2; the first block against the previous call's last), and the
// least-squares sums over the unwrapped delays, x relative to the first block since
// the last reset.  Thread t takes a contiguous run of blocks; the period counts are
// scanned across threads and the sums reduced in a fixed order.
constexpr int kCkThreads = 256;
__device__ __forceinline__ double ck_delay(float2 c, double P)
{
    return -P / (2.0 * 3.14159265358979323846) * atan2((double)c.y, (double)c.x);
}
__global__ void __launch_bounds__(kCkThreads) k_clock_track(const float2 *__restrict__ clk, int nblk, long long b0,
                                                           int N, int P, DevState *dst)
{
    __shared__ int s_k[kCkThreads];
    __shared__ double s_r[4][kCkThreads];
    ClockTrack *ck = &dst->ck;
    const double Pd = (double)P, H = 0.5 * Pd;
    const int t = threadIdx.x, per = (nblk + kCkThreads - 1) / kCkThreads;
    const int lo = min(t * per, nblk), hi = min(lo + per, nblk);
    const int have = ck->have;
    const double dcarry = ck->y - ck->off;   // the previous call's last raw delay
    // period steps: k_i = -1 when d_i - d_{i-1} > P/2, +1 below -P/2
    int ksum = 0;
    double dprev = lo > 0 ? ck_delay(clk[lo - 1], Pd) : dcarry;
    for (int i = lo; i < hi; i++) {
        const double d = ck_delay(clk[i], Pd);
        if (i > 0 || have) ksum += (d - dprev > H) ? -1 : (d - dprev < -H) ? 1 : 0;
        dprev = d;
    }
    s_k[t] = ksum;
    __syncthreads();
    int pre = 0;
    for (int j = 0; j < t; j++) pre += s_k[j];
    const double x0 = ck->n > 0 ? ck->x0 : (double)(N / 2) * (double)b0 + (double)(N / 4);
    const double off0 = have ? ck->off : 0.0;
    double sx = 0, sy = 0, sxx = 0, sxy = 0, ylast = 0, offlast = 0;
    int kk = pre;
    dprev = lo > 0 ? ck_delay(clk[lo - 1], Pd) : dcarry;
    for (int i = lo; i < hi; i++) {
        const double d = ck_delay(clk[i], Pd);
        if (i > 0 || have) kk += (d - dprev > H) ? -1 : (d - dprev < -H) ? 1 : 0;
        dprev = d;
        const double off = off0 + Pd * (double)kk, y = d + off;
        const double x = (double)(N / 2) * (double)(b0 + i) + (double)(N / 4) - x0;
        sx += x;
        sy += y;
        sxx += x * x;
        sxy += x * y;
        ylast = y;
        offlast = off;
    }
    s_r[0][t] = sx;
    s_r[1][t] = sy;
    s_r[2][t] = sxx;
    s_r[3][t] = sxy;
    __syncthreads();
    for (int w = kCkThreads / 2; w > 0; w >>= 1) {
        if (t < w)
            for (int q = 0; q < 4; q++) s_r[q][t] += s_r[q][t + w];
        __syncthreads();
    }
    if (t == 0) {
        ck->x0 = x0;
        ck->sx += s_r[0][0];
        ck->sy += s_r[1][0];
        ck->sxx += s_r[2][0];
        ck->sxy += s_r[3][0];
        ck->n += nblk;
    }
    if (nblk > 0 && hi == nblk && lo < hi) {   // the thread holding the last block
        ck->y = ylast;
        ck->off = offlast;
        ck->have = 1;
    }
}

// self-test of the bounded waits: a phase that nothing completes
__global__ void k_selftest_wait(int *status)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncwarp();
    const bool done = mbar_wait<4096>(&bar, 0);
    if (threadIdx.x == 0) *status = done ? (int)RX_OK : (int)RX_ETIMEOUT;
}

extern "C" {

rx_status rx_selftest_wait_timeout(void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int *d = nullptr, v = -1;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return RX_ECUDA;
    cudaError_t e = cudaMemsetAsync(d, 0xFF, sizeof(int), st);
    if (e == cudaSuccess) {
        k_selftest_wait<<<1, 32, 0, st>>>(d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v, d, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return RX_ECUDA;
    return v == (int)RX_ETIMEOUT ? RX_ETIMEOUT : v == (int)RX_OK ? RX_OK : RX_ECUDA;
}

// 8 independent FMA chains per thread; the sum of the chains goes to *sink
__global__ void __launch_bounds__(256) k_fma_rate(int iters, float a, float b, float *sink)
{
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = fmaf(x[j], a, b);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) s += x[j];
    if (s == 1234.5f) *sink = s;   // practically never; keeps the chains live
}

rx_status rx_selftest_fma_rate(int iters, double *tflops, void *stream)
{
    if (!tflops || iters < 1 || iters > (1 << 24)) return RX_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0, per = 0;
    float *sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    rx_status r = RX_ECUDA;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fma_rate, 256, 0) == cudaSuccess && per > 0 &&
        cudaMalloc(&sink, sizeof(float)) == cudaSuccess && cudaEventCreate(&a) == cudaSuccess &&
        cudaEventCreate(&b) == cudaSuccess) {
        const unsigned grid = (unsigned)(nsm * per);
        // a close to 1, b small: the chains stay finite for any iters
        k_fma_rate<<<grid, 256, 0, st>>>(iters, 0.999999f, 1e-6f, sink);
        cudaEventRecord(a, st);
        k_fma_rate<<<grid, 256, 0, st>>>(iters, 0.999999f, 1e-6f, sink);
        cudaEventRecord(b, st);
        float ms = 0.f;
        if (cudaGetLastError() == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
            cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms > 0.f) {
            *tflops = 16.0 * iters * (double)grid * 256.0 / (ms * 1e-3) / 1e12;
            r = RX_OK;
        }
    }
    cudaGetLastError();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (sink) cudaFree(sink);
    return r;
}

const char *rx_strerror(rx_status s)
{
    switch (s) {
    case RX_OK: return "ok";
    case RX_EINVAL: return "invalid argument or configuration";
    case RX_ENOMEM: return "out of memory";
    case RX_ECUDA: return "CUDA runtime error";
    case RX_ESTATE: return "handle unusable after an earlier failure";
    case RX_ETIMEOUT: return "device-side wait timed out";
    case RX_EBOUNDS: return "output capacity too small";
    }
    return "unknown status";
}

rx_status rx_default_config(rx_format f, rx_config *c)
{
    if (!c || (int)f < 0 || (int)f > 4) return RX_EINVAL;
    memset(c, 0, sizeof *c);
    int kk = f >= RX_KK_QPSK;
    c->pack_order = 0;
    c->ols_n = kk ? 65536 : 0;
    c->ols_v = kk ? 4096 : 0;
    c->ds_num = kk ? 11 : 0;
    c->ds_den = kk ? 80 : 1;
    c->rrc_beta = 0.1;
    c->mf_span = 16;
    c->ntaps = kk ? 31 : 15;
    c->ntrain = kk ? 16384 : 4096;
    c->ncma = kk ? 8192 : 0;
    // the paper's 8192 data blocks of a 2^22-sample buffer: 128 symbols at 4 samples/symbol
    // (KK), 256 at 2 samples/symbol (PAM)
    c->eq_block = kk ? 128 : 256;
    c->win = 64;
    c->mu = 1e-3;
    c->mu_train = 1e-3;
    c->mu_cma = 1e-3;
    c->bps_b = 32;
    c->amb_syms = kk ? 1024 : 0;
    c->prbs_seed = 1;
    c->debug = 0;
    c->mf_mode = RX_MF_TIME;
    c->fd_n = 1024;
    c->fd_taps = kk ? 203 : 503;
    c->cnn_bf16 = 1;
    return RX_OK;
}

int64_t rx_max_bits(const rx_handle *h)
{
    if (!h) return 0;
    long long call = (long long)h->bps * (h->nb / h->sps + h->cfg.eq_block + h->cfg.ntrain + 64);
    return call > h->flush_bits ? call : h->flush_bits;
}

void rx_destroy(rx_handle *h)
{
    if (!h) return;
    // work still queued on the pipeline's own streams finishes before the memory goes
    if (h->front) cudaStreamSynchronize(h->front);
    if (h->front2) cudaStreamSynchronize(h->front2);
    if (h->mid) cudaStreamSynchronize(h->mid);
    if (h->back) cudaStreamSynchronize(h->back);
    if (h->tail) cudaStreamSynchronize(h->tail);
    if (h->copy) cudaStreamSynchronize(h->copy);
    void *ptrs[] = {h->codes[0], h->codes[1], h->fftws[0], h->fftws[1], h->prbs, h->taps[0], h->taps[1], h->twN,
                    h->twN2, h->ds_tab, h->rrc, h->dbg_win, h->dbg_z, h->st,
                    h->bits_stage, h->lnt, h->prbs_bits, h->phist[0], h->phist[1], h->phist[2], h->zbuf, h->gpart, h->fd_H, h->fd_tw, h->R[0], h->R[1],
                    h->rs_tab, h->clk, h->lat_dev};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (int i = 0; i < kSlots; i++) {
        void *sp[] = {h->E[i], h->Y[i], h->dec[i], h->winb[i], h->winrec[i]};
        for (void *p : sp)
            if (p) cudaFree(p);
        cudaEvent_t ev[] = {h->ev_yfree[i], h->ev_efree[i], h->ev_dfree[i]};
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
    if (h->prof_ev) {
        for (int i = 0; i < kProfRing * kEvPerCall; i++) cudaEventDestroy(h->prof_ev[i]);
        free(h->prof_ev);
    }
    free(h->lat_hist);
    if (h->front) cudaStreamDestroy(h->front);
    if (h->front2) cudaStreamDestroy(h->front2);
    if (h->mid) cudaStreamDestroy(h->mid);
    if (h->back) cudaStreamDestroy(h->back);
    if (h->tail) cudaStreamDestroy(h->tail);
    if (h->copy) cudaStreamDestroy(h->copy);
    cudaEvent_t *evs[] = {&h->ev_fork, &h->ev_front, &h->ev_hist, &h->ev_join, &h->ev_cfree[0], &h->ev_cfree[1]};
    for (cudaEvent_t *ev : evs)
        if (*ev) cudaEventDestroy(*ev);
    for (int i = 0; i < kInSlots; i++) {
        if (h->ev_inready[i]) cudaEventDestroy(h->ev_inready[i]);
        if (h->ev_infree[i]) cudaEventDestroy(h->ev_infree[i]);
        if (h->in_stage[i]) cudaFree(h->in_stage[i]);
    }
    free(h->prof_used);
    free(h);
}

#define RX_ALLOC(ptr, bytes)                                                            \
    do {                                                                                \
        if (cudaMalloc((void **)&(ptr), (size_t)(bytes)) != cudaSuccess) {              \
            cudaGetLastError();                                                         \
            rx_destroy(h);                                                              \
            return RX_ENOMEM;                                                           \
        }                                                                               \
        if (cudaMemset((ptr), 0, (size_t)(bytes)) != cudaSuccess) {                     \
            rx_destroy(h);                                                              \
            return RX_ECUDA;                                                            \
        }                                                                               \
    } while (0)

// Response of the zero-phase taps h_i = re[i + L] + j im[i + L], i = -L .. L, at the
// bins the frequency-domain kernels multiply, times 1/N: KK the N/2 kept bins in
// downsampled order (k' < N/4 -> k = k', else k = k' + N/2), PAM all N bins.
static void fd_response(const double *re, const double *im, int ntaps, int N, bool kk, float2 *Hk)
{
    const double pi = 3.14159265358979323846;
    const int half = (ntaps - 1) / 2, nbins = kk ? N / 2 : N;
    for (int kp = 0; kp < nbins; kp++) {
        const int k = (!kk || kp < N / 4) ? kp : kp + N / 2;
        double hr = 0, hi = 0;
        for (int i = -half; i <= half; i++) {
            const double a = -2.0 * pi * (double)(((long long)k * i) % N) / N;
            const double tr = re[i + half], ti = im ? im[i + half] : 0.0;
            hr += tr * cos(a) - ti * sin(a);
            hi += tr * sin(a) + ti * cos(a);
        }
        Hk[kp] = make_float2((float)(hr / N), (float)(hi / N));
    }
}

rx_status rx_create(rx_format f, double baud, double fs, int64_t buf_len, const rx_config *cfg_in,
                    rx_handle **out)
{
    if (!out) return RX_EINVAL;
    *out = nullptr;
    if ((int)f < 0 || (int)f > 4 || !(baud > 0) || !(fs > 0) || buf_len <= 0 || buf_len % 32) return RX_EINVAL;
    rx_config c;
    if (cfg_in) c = *cfg_in;
    else rx_default_config(f, &c);
    int kk = f >= RX_KK_QPSK;
    double ratio = fs / baud;
    int sps = (int)floor(ratio + 0.5);
    if (fabs(ratio - sps) > 1e-9 * ratio || sps != (kk ? 4 : 2)) return RX_EINVAL;
    if (c.eq_mode < RX_EQ_WINDOW || c.eq_mode > RX_EQ_DD_SYMBOL ||
        (c.eq_mode == RX_EQ_DD_SYMBOL && (!kk || c.ntaps < 2 || c.ntaps > 8 || c.fir_prec != RX_FIR_ADAPTIVE)))
        return RX_EINVAL;
    if (c.pack_order < 0 || c.pack_order > 1 || c.ntaps < 1 || c.ntaps > kMaxTaps ||
        (!(c.ntaps & 1) && c.eq_mode != RX_EQ_DD_SYMBOL) ||
        c.win != kWin || c.eq_block < kWin || c.eq_block % kWin || c.ntrain < 0 || c.ntrain % kWin ||
        c.mf_span < 0 || c.mf_span % 2 || sps * c.mf_span / 2 > kEHist / 2 || !(c.rrc_beta >= 0) ||
        c.rrc_beta > 1 || c.eq_block > kMaxEqBlock)
        return RX_EINVAL;
    if (c.fir_prec < RX_FIR_ADAPTIVE || c.fir_prec > RX_FIR_FP8 || (c.fir_prec != RX_FIR_ADAPTIVE && !kk) ||
        (c.fir_prec >= RX_FIR_BF16 && 2048 % c.eq_block))
        return RX_EINVAL;
    if (c.kk_front < 0 || c.kk_front > 1 || !(c.eq_warps == 0 || c.eq_warps == 2 || c.eq_warps == 4 || c.eq_warps == 8))
        return RX_EINVAL;
    if (c.rs_step != 0 && ((!kk && c.mf_mode == RX_MF_FD) || c.rs_step < 4252017623LL || c.rs_step > 4337916969LL))
        return RX_EINVAL;
    if (c.cnn_bf16 < 0 || c.cnn_bf16 > 1 || !(c.deadline_ms == c.deadline_ms)) return RX_EINVAL;
    if (c.diff_code < 0 || c.diff_code > 1 || (c.diff_code && !kk)) return RX_EINVAL;
    if (c.clk_track < 0 || c.clk_track > 1 || (c.clk_track && c.mf_mode != RX_MF_FD)) return RX_EINVAL;
    if (c.mf_mode < RX_MF_TIME || c.mf_mode > RX_MF_FD ||
        (c.mf_mode == RX_MF_FD && (c.fd_n < 16 || c.fd_n > kEHist || (c.fd_n & (c.fd_n - 1)) ||
                                   (!kk && c.fd_n != 1024) || c.fd_taps < 1 || !(c.fd_taps & 1) ||
                                   c.fd_taps > c.fd_n / 2 + 1)))
        return RX_EINVAL;
    if (kk && (c.ncma < 0 || c.ncma > c.ntrain || c.ncma % kWin || c.bps_b < 1 || c.bps_b > 32 ||
               c.ds_den < 1 || c.ds_num < 0 || c.amb_syms < 0 || c.amb_syms % kWin || c.amb_syms > 4096 ||
               !(c.ols_n == 4096 || c.ols_n == 65536) || c.ols_v < 64 || c.ols_v % 64 || c.ols_v >= c.ols_n))
        return RX_EINVAL;
    // size limits: per-call symbol and window counts are 32-bit, and the KK forward
    // pass has one grid row per overlap-save block pair plus the history copy (<= 65535)
    if (buf_len > (1LL << 30)) return RX_EINVAL;
    if (kk) {
        const long long hop = c.ols_n - c.ols_v, jmax = (buf_len + hop - 1) / hop + 1;
        if ((jmax + 1) / 2 + 1 > 65535) return RX_EINVAL;
    }
    rx_handle *h = (rx_handle *)calloc(1, sizeof(rx_handle));
    if (!h) return RX_ENOMEM;
    h->fmt = f;
    h->kk = kk;
    h->bps = (f == RX_PAM2) ? 1 : (f == RX_PAM4) ? 2 : (f == RX_PAM8) ? 3 : (f == RX_KK_QPSK) ? 2 : 4;
    h->mq = kk ? ((f == RX_KK_QPSK) ? 2 : 4) : (1 << h->bps);
    h->sps = sps;
    h->decim = sps / 2;
    h->hmf = sps * c.mf_span / 2;
    h->fd = c.mf_mode == RX_MF_FD;
    h->rs = c.rs_step != 0;
    h->th = (c.ntaps - 1) / 2;
    h->nb = buf_len;
    h->cfg = c;
    h->nhist = kk ? c.ols_n : (c.mf_mode == RX_MF_FD ? c.fd_n : kPamHist);
    if (kk) {
        h->N = c.ols_n;
        h->V = c.ols_v;
        h->hop = h->N - h->V;
        h->N2 = h->N / 16;
        long long jmax = (buf_len + h->hop - 1) / h->hop + 1;
        h->npairs_max = (int)((jmax + 1) / 2);
    }
    EqParams &p = h->ep;
    p.kk = kk;
    p.mq = h->mq;
    p.bps = h->bps;
    p.ntaps = c.ntaps;
    p.dd = c.eq_mode == RX_EQ_DD_SYMBOL;
    p.th = h->th;
    p.win = c.win;
    p.eq_block = c.eq_block;
    p.ntrain = c.ntrain;
    p.ncma = c.ncma;
    p.bps_b = c.bps_b;
    p.amb_syms = c.amb_syms;
    p.scale = kk ? (float)((f == RX_KK_QPSK) ? sqrt(2.0) : sqrt(10.0)) : 1.f;
    p.r2 = kk ? ((f == RX_KK_QPSK) ? 1.f : 1.32f) : 0.f;
    p.mu = (float)c.mu;
    p.mu_train = (float)c.mu_train;
    p.mu_cma = (float)c.mu_cma;
    p.frozen = c.fir_prec != RX_FIR_ADAPTIVE;
    p.diff = c.diff_code;
    if (c.eq_warps) {
        p.warps = c.eq_warps;
        if (eq_smem_bytes(p, p.warps) > kMaxSmemCta) { free(h); return RX_EINVAL; }
    } else {   // default: 4 blocks per CTA, fewer when long blocks do not fit
        p.warps = 4;
        while (p.warps > 1 && eq_smem_bytes(p, p.warps) > kMaxSmemCta) p.warps /= 2;
    }

    // the first call that emits payload must carry the ambiguity-resolution symbols
    if (kk && c.amb_syms > 0) {
        long long qp = 0;
        for (long long k = 0; k < (1 << 20); k++) {
            Sched s = schedule(h, k, qp);
            if (s.q_k > c.ntrain) {   // first call that emits payload
                if (s.q_k - (qp > c.ntrain ? qp : c.ntrain) < c.amb_syms) { free(h); return RX_EINVAL; }
                break;
            }
            qp = s.q_k;
        }
    }

    // bound of the payload symbols rx_flush emits: the largest lag of the schedule
    // (symbols of the stream not yet decided after a call), over enough calls to
    // pass training and reach the steady state
    {
        long long qp = 0, lag = 0;
        long long span = (long long)c.ntrain * sps + (kk ? c.ols_n : 0) + (long long)c.eq_block * sps + 8192;
        long long ncalls = 64 + 8 * span / buf_len;
        if (ncalls > 200000) ncalls = 200000;
        for (long long k = 0; k < ncalls; k++) {
            Sched s = schedule(h, k, qp);
            long long l = (k + 1) * buf_len / sps - s.q_k;
            if (l > lag) lag = l;
            qp = s.q_k;
        }
        if (h->rs) lag += buf_len / 50 / sps + 16;   // nominal grid within 1 % of the ADC's
        h->flush_bits = (long long)h->bps * (lag + 64);
    }
    long long nb = buf_len;
    long long symcap = nb / sps + 2LL * c.eq_block + c.ntrain + 256;
    h->dec_cap = symcap;
    h->win_cap = symcap / kWin + 1;
    h->y_cap = nb / h->decim + 2LL * c.eq_block + 2LL * c.ntrain + 256;
    size_t yel = kk ? sizeof(float2) : sizeof(float);
    for (int i = 0; i < 2; i++) {
        RX_ALLOC(h->codes[i], (h->nhist + nb) * sizeof(uint16_t));
        RX_ALLOC(h->taps[i], 32 * sizeof(float2));
    }
    for (int i = 0; i < kSlots; i++) {
        RX_ALLOC(h->Y[i], h->y_cap * yel);
        RX_ALLOC(h->dec[i], h->dec_cap);
        RX_ALLOC(h->winb[i], h->win_cap);
        RX_ALLOC(h->winrec[i], h->win_cap * sizeof(uint4));
    }
    if (kk) {
        for (int i = 0; i < kSlots; i++) RX_ALLOC(h->E[i], (kEHist + nb) * sizeof(float2));
        for (int i = 0; i < 3; i++) RX_ALLOC(h->phist[i], (size_t)h->nhist * 3 / 2 + 16);
        for (int i = 0; i < 2; i++) RX_ALLOC(h->fftws[i], (size_t)h->npairs_max * h->N * sizeof(float2));
        RX_ALLOC(h->twN, kk_tw_entries(h->N) * sizeof(float2));
        RX_ALLOC(h->twN2, kk_tw_entries(h->N2) * sizeof(float2));
        RX_ALLOC(h->lnt, kLutCodes * sizeof(float));
        RX_ALLOC(h->ds_tab, c.ds_den * sizeof(float2));
    }
    if (h->rs) {   // a call emits at most nb / 0.99 + 8 nominal samples
        for (int i = 0; i < 2; i++) RX_ALLOC(h->R[i], (kEHist + nb + nb / 64 + 64) * sizeof(float2));
        RX_ALLOC(h->rs_tab, 1024 * 16 * sizeof(float));
        if (!kk) RX_ALLOC(h->E[0], (h->nhist + nb) * sizeof(float2));   // PAM: the normalised codes
    }
    RX_ALLOC(h->prbs, 32767 + 256);
    RX_ALLOC(h->prbs_bits, kPrbsWords * sizeof(uint32_t));
    RX_ALLOC(h->rrc, (2 * h->hmf + 1) * sizeof(float));
    RX_ALLOC(h->st, sizeof(DevState));
    for (int i = 0; i < kInSlots; i++) RX_ALLOC(h->in_stage[i], nb * 3 / 2 + 16);
    RX_ALLOC(h->bits_stage, rx_max_bits(h) / 8 + 16);
    if (c.fir_prec >= RX_FIR_BF16) RX_ALLOC(h->zbuf, symcap * sizeof(float2));
    if (c.fir_prec >= RX_FIR_FROZEN_F32) RX_ALLOC(h->gpart, (size_t)(kMaxEqBlock / kWin) * 32 * sizeof(float2));
    if (c.debug) {
        RX_ALLOC(h->dbg_win, h->win_cap * sizeof(float4));
        RX_ALLOC(h->dbg_z, symcap * sizeof(float2));
    }

    // constant tables (host double precision, rounded once)
    int nt = 2 * h->hmf + 1;
    double *hd = (double *)malloc(sizeof(double) * nt);
    float *hf = (float *)malloc(sizeof(float) * nt);
    rrc_taps(c.rrc_beta, sps, c.mf_span, hd);
    for (int i = 0; i < nt; i++) hf[i] = (float)hd[i];
    for (int i = 0; i < nt && i < (int)(sizeof h->rrc_host / sizeof(float)); i++) h->rrc_host[i] = hf[i];
    cudaError_t e = cudaMemcpy(h->rrc, hf, sizeof(float) * nt, cudaMemcpyHostToDevice);
    free(hd);
    free(hf);
    uint8_t *pb = (uint8_t *)malloc(32767 + 256);
    prbs15_period(c.prbs_seed, pb);
    for (int i = 0; i < 256; i++) pb[32767 + i] = pb[i];   // one period plus its first 256 bits again
    if (e == cudaSuccess) e = cudaMemcpy(h->prbs, pb, 32767 + 256, cudaMemcpyHostToDevice);
    uint32_t pw[kPrbsWords];
    memset(pw, 0, sizeof pw);
    for (int i = 0; i < 32767 + 256; i++)
        if (pb[i]) pw[i >> 5] |= 0x80000000u >> (i & 31);
    if (e == cudaSuccess) e = cudaMemcpy(h->prbs_bits, pw, sizeof pw, cudaMemcpyHostToDevice);
    free(pb);
    float2 t0[32];
    memset(t0, 0, sizeof t0);
    t0[h->th] = make_float2(1.f, 0.f);   // centre tap 1
    if (e == cudaSuccess) e = cudaMemcpy(h->taps[0], t0, sizeof t0, cudaMemcpyHostToDevice);
    if (kk && e == cudaSuccess) {
        int n1 = kk_tw_entries(h->N), n2 = kk_tw_entries(h->N2);
        float2 *t1 = (float2 *)malloc(sizeof(float2) * n1), *t2 = (float2 *)malloc(sizeof(float2) * n2);
        float *ln = (float *)malloc(sizeof(float) * kLutCodes);
        kk_host_tables(h->N, ln, t1, t2);
        e = cudaMemcpy(h->twN, t1, sizeof(float2) * n1, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->twN2, t2, sizeof(float2) * n2, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->lnt, ln, sizeof(float) * kLutCodes, cudaMemcpyHostToDevice);
        free(t1);
        free(t2);
        free(ln);
        float2 *ds = (float2 *)malloc(sizeof(float2) * c.ds_den);
        twiddles(c.ds_den, ds);      // e^{-2 pi i p / den}
        if (e == cudaSuccess) e = cudaMemcpy(h->ds_tab, ds, sizeof(float2) * c.ds_den, cudaMemcpyHostToDevice);
        free(ds);
    }
    if (h->fd) {
        // frequency-domain filter: response of the zero-phase RRC taps at the kept
        // bins, times 1/N; N-point twiddles
        const int N = c.fd_n, half = (c.fd_taps - 1) / 2, nbins = kk ? N / 2 : N;
        double *hf = (double *)malloc(sizeof(double) * c.fd_taps);
        float2 *Hk = (float2 *)malloc(sizeof(float2) * nbins), *tw = (float2 *)malloc(sizeof(float2) * N);
        rrc_half(c.rrc_beta, sps, half, hf);
        fd_response(hf, nullptr, c.fd_taps, N, kk, Hk);
        twiddles(N, tw);
        // band-edge clock correlation per block: half-width ceil(beta S / 2) bins around
        // S / 2, S = N / sps the bin of the symbol rate (the 1024-point kernels cover 31)
        if (kk) {   // blocks per call: nominal samples (nb / 0.99 + 8 with the resampler) / (N/2) + 2
            h->clk_w = (int)ceil(c.rrc_beta * N / 8.0);
            if (h->clk_w >= N / 8) h->clk_w = N / 8 - 1;
            if (N == 1024 && h->clk_w > 31) h->clk_w = 31;
            if (e == cudaSuccess) e = cudaMalloc(&h->clk, sizeof(float2) * ((nb + nb / 64 + 64) / (N / 2) + 4));
        } else {    // PAM: N = 1024 at 2 samples/symbol, N / 2 outputs per block
            h->clk_w = (int)ceil(c.rrc_beta * N / 4.0);
            if (h->clk_w > 31) h->clk_w = 31;
            if (e == cudaSuccess) e = cudaMalloc(&h->clk, sizeof(float2) * (nb / (N / 2) + 4));
        }
        if (e == cudaSuccess) e = cudaMalloc(&h->fd_H, sizeof(float2) * nbins);
        if (e == cudaSuccess) e = cudaMalloc(&h->fd_tw, sizeof(float2) * N);
        if (e == cudaSuccess) e = cudaMemcpy(h->fd_H, Hk, sizeof(float2) * nbins, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->fd_tw, tw, sizeof(float2) * N, cudaMemcpyHostToDevice);
        free(hf);
        free(Hk);
        free(tw);
    }
    if (h->rs) {
        // interpolator taps c_j(q / 1024) = sinc(j - mu) (1 + cos(pi (j - mu) / 8)) / 2, j = -7..8
        const double pi = 3.14159265358979323846;
        float *tab = (float *)malloc(sizeof(float) * 1024 * 16);
        for (int q = 0; q < 1024; q++)
            for (int j = -7; j <= 8; j++) {
                double x = (double)j - q / 1024.0;
                double sn = fabs(x) < 1e-15 ? 1.0 : sin(pi * x) / (pi * x);
                double w = fabs(x) < 8.0 ? 0.5 * (1.0 + cos(pi * x / 8.0)) : 0.0;
                tab[q * 16 + j + 7] = (float)(sn * w);
            }
        if (e == cudaSuccess) e = cudaMemcpy(h->rs_tab, tab, sizeof(float) * 1024 * 16, cudaMemcpyHostToDevice);
        free(tab);
    }
    DevState s0;
    memset(&s0, 0, sizeof s0);
    for (int i = 0; i < kSlots; i++) s0.cg[i][2] = 1.0;
    s0.amb_r = -1;
    if (e == cudaSuccess) e = cudaMemcpy(h->st, &s0, sizeof s0, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        rx_destroy(h);
        return RX_ECUDA;
    }
    h->rs_r0 = 0;
    h->rs_psi0 = (__int128)c.rs_phase0;
    h->ebase_cur = -kEHist;
    h->rbase_cur = -kEHist;
    h->ybase_cur = -kYHist;
    {
        // one priority for every stage: measured against the field and matched filter
        // ahead of the back end, and against the equaliser (the longest chain from
        // buffer to buffer) ahead of the rest, equal priorities gave the highest
        // throughput with device and with host buffers
        bool ok = cudaStreamCreateWithFlags(&h->front, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&h->front2, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&h->mid, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&h->back, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&h->tail, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&h->copy, cudaStreamNonBlocking) == cudaSuccess;
        cudaEvent_t *evs[] = {&h->ev_fork, &h->ev_front, &h->ev_hist, &h->ev_join, &h->ev_cfree[0], &h->ev_cfree[1]};
        for (cudaEvent_t *ev : evs)
            ok = ok && cudaEventCreateWithFlags(ev, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; i < kInSlots; i++)
            ok = ok && cudaEventCreateWithFlags(&h->ev_inready[i], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&h->ev_infree[i], cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; i < kSlots; i++)
            ok = ok && cudaEventCreateWithFlags(&h->ev_yfree[i], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&h->ev_efree[i], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&h->ev_dfree[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            rx_destroy(h);
            return RX_ECUDA;
        }
    }
    if (c.deadline_ms >= 0) {
        h->lat_budget = c.deadline_ms > 0 ? c.deadline_ms : 5.0 * (double)buf_len / fs * 1e3;
        h->lat_hist = (uint32_t *)calloc(kLatBins, sizeof(uint32_t));
        const unsigned long long budget_ns = (unsigned long long)llround(h->lat_budget * 1e6);
        bool ok = h->lat_hist && cudaMalloc(&h->lat_dev, sizeof(LatRecord)) == cudaSuccess &&
                  cudaMemset(h->lat_dev, 0, sizeof(LatRecord)) == cudaSuccess &&
                  cudaMemcpy(&h->lat_dev->budget_ns, &budget_ns, sizeof budget_ns, cudaMemcpyHostToDevice) ==
                      cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            rx_destroy(h);
            return RX_ECUDA;
        }
    }
    {
        int dev = 0;
        bool ok = cudaGetDevice(&dev) == cudaSuccess &&
                  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                  prepare_eq(h->ep) == cudaSuccess && (!kk || prepare_kk_front() == cudaSuccess) &&
                  (c.fir_prec < RX_FIR_BF16 || prepare_fir_tc(c.fir_prec) == cudaSuccess);
        if (!ok) {
            cudaGetLastError();
            rx_destroy(h);
            return RX_ECUDA;
        }
    }
    *out = h;
    return RX_OK;
}

// Enqueue one buffer: field reconstruction and matched filter on `sf`, equaliser,
// decisions and bits on `sb` (the same stream for rx_process).  With two streams
// the back end of this call waits for its front end, and the front end of a later
// call that reuses a matched-filter slot waits for the back end that read it.
// With host buffers (host_in / host_out non-null) the input is copied into one of
// two staging buffers on `sc`, overlapping the previous front end, and the bits
// are copied back on `sb` after the demap.
static rx_status enqueue_call(rx_handle *h, const uint8_t *in, uint8_t *bits_out, const uint8_t *host_in,
                              uint8_t *host_out, cudaStream_t sf, cudaStream_t sb, cudaStream_t sc,
                              int64_t *nbits_out, cudaStream_t smid = nullptr, cudaStream_t stail = nullptr)
{
    const rx_config &c = h->cfg;
    Sched s = schedule(h, h->calls, h->q_prev);
    long long base = h->calls * h->nb;
    long long sym_lo = h->trained ? h->q_prev : 0;
    bool do_train = !h->trained && s.q_k >= c.ntrain && s.q_k > 0;
    long long pay_lo = do_train ? c.ntrain : h->q_prev;
    long long npay = (h->trained || do_train) ? s.q_k - pay_lo : 0;
    if (npay > 0 && !bits_out && !host_out) return RX_EINVAL;
    // latency record of calls that emit payload (not inside group rounds or flushes):
    // the call's first kernel stamps its slot, its demap closes it
    const bool lat = h->lat_dev && !h->in_group && !h->flush_mode && npay >= c.eq_block;
    const int lat_slot = (int)(h->lat_head % kLatSlots);
    LatRecord *lat_first = lat ? h->lat_dev : nullptr;
    // the launchers detect failures with cudaGetLastError: clear an error some
    // earlier, unrelated call left behind (a sticky one makes the launches fail)
    cudaError_t stale = cudaGetLastError();
    if (stale != cudaSuccess) traced(stale, "an earlier CUDA call (cleared)");
    const bool two = sf != sb;
    // in the pipeline the filter runs on a third stream between the front end (KK field,
    // PAM unpack) and the equaliser (back); field and codes slots wait for it to be done
    const bool three = two && smid;
    cudaStream_t sm = three ? smid : sf;
    // the demap (and the copy of the bits) on a fourth stream, after its equaliser
    const bool four = two && stail;
    cudaStream_t st4 = four ? stail : sb;
    cudaError_t e = cudaSuccess;
    int par = (int)(h->calls & 1);
    const int isl = (int)(h->calls % kInSlots);   // input staging slot of a host-buffer call
    const int spar = (int)(h->calls % 3);   // PAM sums slot: the filter of call i clears call i+2's
    int ds = (int)(h->calls % kSlots);   // decision slot of this call
    // KK in the pipeline: the field of odd calls on the second front-end stream.
    // Not with the CNN receiver: its decision kernel is persistent (one CTA per SM),
    // and a second field in flight holds SMs it waits for.
    const bool alt = three && h->kk && h->front2 && !h->cnn;
    if (alt && par) sf = h->front2;
    const KkSync ksync = {alt ? h->ev_hist : nullptr, alt ? h->ev_hist : nullptr, alt ? h->ev_front : nullptr};
    if (host_in) {
        in = h->in_stage[isl];
        if (sc != sf) cudaStreamWaitEvent(sc, h->ev_infree[isl], 0);   // the front end kInSlots calls back is done
        e = cudaMemcpyAsync(h->in_stage[isl], host_in, (size_t)(h->nb * 3 / 2), cudaMemcpyHostToDevice, sc);
        if (sc != sf) {
            cudaEventRecord(h->ev_inready[isl], sc);
            cudaStreamWaitEvent(sf, h->ev_inready[isl], 0);
        }
    }
    if (host_out) bits_out = h->bits_stage;

    h->prof_cur = h->prof_on > 0 && h->calls % h->prof_on == 0;
    if (h->prof_cur && h->prof_head - h->prof_tail >= kProfRing) prof_harvest_one(h);
    // 12-bit unpack into [history | buffer]: the PAM chain's input; the KK kernels
    // read the packed bytes themselves, so there it only feeds the debug view
    if (!h->kk || c.debug) {
        prof_begin(h, 0, sf);
        int cw_new = h->cw ^ 1;
        // PAM in the pipeline: the filter two calls back (on its own stream) is done with
        // this codes slot, and has cleared this call's sums
        if (three && !h->kk) cudaStreamWaitEvent(sf, h->ev_cfree[cw_new], 0);
        // a flush pad adds nothing to the PAM sums: its filter uses the last real buffer's
        const bool sums = !h->kk && !h->flush_mode;
        e = launch_unpack(in, h->codes[cw_new], h->codes[h->cw], h->nb, h->nhist, h->nb, h->calls == 0,
                          c.pack_order, sums ? &h->st->pam_s1[spar] : nullptr,
                          sums ? &h->st->pam_s2[spar] : nullptr, sf, lat_first, lat_slot);
        lat_first = nullptr;   // stamped: the KK front end (debug view) comes after
        h->cw = cw_new;
        prof_end(h, 0, sf);
    }
    KkInput kin;
    if (h->kk) {
        kin.hist = h->phist[h->hw];
        kin.in = in;
        kin.hist_next = h->phist[(h->hw + 1) % 3];
        kin.hist_bytes = (long long)h->nhist * 3 / 2;
        kin.in_bytes = h->nb * 3 / 2;
        kin.order = c.pack_order;
        kin.first_call = h->calls == 0;
        kin.lat = lat_first;
        kin.lat_slot = lat_slot;
    }
    long long cbase = base - h->nhist;

    // KK field reconstruction
    if (e == cudaSuccess && h->kk && s.e_k > h->e_prev) {
        KkGeom g;
        g.e_prev = h->e_prev;
        g.e_k = s.e_k;
        g.avail = s.avail;
        g.cbase = cbase;
        g.ebase = h->e_prev - kEHist;
        g.ebase_prev = h->ebase_cur;
        g.N = h->N;
        g.V = h->V;
        g.hop = h->hop;
        g.J = (int)((s.e_k - h->e_prev + h->hop - 1) / h->hop);
        g.npairs = (g.J + 1) / 2;
        g.N2 = h->N2;
        g.sps = h->sps;
        int ew_new = (h->ew + 1) % kSlots;
        g.slot = ew_new;
        g.fused = c.kk_front;
        if (three) cudaStreamWaitEvent(sf, h->ev_efree[ew_new], 0);   // the matched filter is done with this slot
        KkTables tb = {h->lnt, h->twN, h->twN2};
        e = traced(launch_kk_front(g, kin, h->fftws[par], tb, h->E[ew_new], h->E[h->ew], h->st, sf,
                                   h->prof_cur ? h : nullptr, ksync), "KK front end");
        h->ew = ew_new;
        h->ebase_cur = g.ebase;
    } else if (e == cudaSuccess && h->kk) {
        e = traced(launch_kk_hist(kin, sf, ksync), "KK history copy");
    }
    if (h->kk) h->hw = (h->hw + 1) % 3;
    if (three) {
        if (host_in && sc != sf) cudaEventRecord(h->ev_infree[isl], sf);   // the field has read the input
        cudaEventRecord(h->ev_front, sf);
        cudaStreamWaitEvent(sm, h->ev_front, 0);
    }
    // matched filter (after the resampler when the ADC clock is not the transmitter's)
    prof_begin(h, 4, sm);
    if (e == cudaSuccess && h->rs && s.r_k > h->r_prev) {
        const __int128 psi = rs_psi(h, h->r_prev);
        const long long rb = h->r_prev - kEHist;
        const int ppar_rs = h->flush_mode ? h->flush_par : spar;
        // the resampler reads the reconstructed field (KK) or the call's normalised codes (PAM)
        if (!h->kk) e = launch_pam_norm(h->codes[h->cw], cbase, h->nb, s.avail, h->st, ppar_rs, h->E[0], sm);
        if (e == cudaSuccess)
            e = launch_kk_resample(h->kk ? h->E[h->ew] : h->E[0], h->kk ? h->ebase_cur : cbase, h->r_prev, s.r_k,
                                   (long long)(psi >> 32), (unsigned)(psi & 0xFFFFFFFF), c.rs_step, h->rs_tab,
                                   h->R[h->rw ^ 1], rb, h->R[h->rw], h->rbase_cur, sm);
        h->rw ^= 1;
        h->rbase_cur = rb;
    }
    if (e == cudaSuccess && s.f_k > h->f_prev) {
        long long yb = 2 * h->q_prev - kYHist;
        int yw_new = (h->yw + 1) % kSlots;
        if (two) cudaStreamWaitEvent(sm, h->ev_yfree[yw_new], 0);   // the back end is done with this slot
        // the filter reads the field on the transmitter's grid: resampled, or as reconstructed
        const float2 *Ef = h->kk && h->rs ? h->R[h->rw] : h->E[h->ew];
        // carrier and gain of this call (of the last real buffer in a flush)
        const double *cgp = h->flush_mode ? h->st->cg_flush : &h->st->cg[h->ew][0];
        const int ppar = h->flush_mode ? h->flush_par : spar;
        const long long efbase = h->kk && h->rs ? h->rbase_cur : h->ebase_cur;
        if (h->kk && h->fd)
            e = launch_kk_fdmf(Ef, efbase, h->f_prev, s.f_k, c.fd_n, h->fd_H, h->fd_tw, h->ds_tab,
                               c.ds_num, c.ds_den, cgp, (float2 *)h->Y[yw_new], yb,
                               (const float2 *)h->Y[h->yw], h->ybase_cur, sm, h->clk, h->clk_w);
        else if (h->kk)
            e = launch_kk_mf(Ef, efbase, s.r_k, h->f_prev, s.f_k, h->rrc, h->hmf, h->ds_tab, c.ds_num,
                             c.ds_den, cgp, (float2 *)h->Y[yw_new], yb, (const float2 *)h->Y[h->yw],
                             h->ybase_cur, sm, h->rrc_host);
        else if (h->rs)
            e = launch_pam_mf_r(h->R[h->rw], h->rbase_cur, h->f_prev, s.f_k, h->rrc, h->hmf, (float *)h->Y[yw_new], yb,
                                (const float *)h->Y[h->yw], h->ybase_cur, sm);
        else if (h->fd)
            e = launch_pam_fd1024(h->codes[h->cw], cbase, h->nb, s.avail, h->f_prev, s.f_k, h->fd_H, h->fd_tw, h->st,
                                  ppar, (float *)h->Y[yw_new], yb, (const float *)h->Y[h->yw], h->ybase_cur, sm,
                                  h->clk, h->clk_w);
        else
            e = launch_pam_mf(h->codes[h->cw], cbase, h->nb, s.avail, h->f_prev, s.f_k, h->rrc, h->hmf, h->st, ppar,
                              (float *)h->Y[yw_new], yb, (const float *)h->Y[h->yw], h->ybase_cur, sm);
        if (e == cudaSuccess && h->fd && c.clk_track) {
            // blocks of this call: outputs at 2 samples/symbol per block N/4 (KK) or N/2 (PAM)
            const long long per = h->kk ? c.fd_n / 4 : c.fd_n / 2;
            const long long nblk = (s.f_k - h->f_prev) / per;
            if (nblk > 0) {
                k_clock_track<<<1, kCkThreads, 0, sm>>>(h->clk, (int)nblk, h->f_prev / per, c.fd_n,
                                                                    h->sps, h->st);
                e = cudaGetLastError();
            }
        }
        h->yw = yw_new;
        h->ybase_cur = yb;
    }
    prof_end(h, 4, sm);
    if (three) {
        // the field (KK) or codes (PAM) slot's release is also the equaliser's start signal
        cudaEvent_t rel = h->kk ? h->ev_efree[h->ew] : h->ev_cfree[h->cw];
        cudaEventRecord(rel, sm);
        cudaStreamWaitEvent(sb, rel, 0);
    } else {
        if (host_in && sc != sf) cudaEventRecord(h->ev_infree[isl], sf);
        if (two) {
            cudaEventRecord(h->ev_front, sf);
            cudaStreamWaitEvent(sb, h->ev_front, 0);
        }
    }
    // equaliser, decisions, bits
    EqGeom g;
    memset(&g, 0, sizeof g);
    g.sym_lo = sym_lo;
    g.pay_lo = pay_lo;
    g.q_k = s.q_k;
    g.ybase = h->ybase_cur;
    g.nblk = npay > 0 ? (int)(npay / c.eq_block) : 0;
    g.nwin = npay > 0 ? (int)(npay / kWin) : 0;
    g.gpart = h->gpart;
    g.score_end = h->flush_mode ? h->flush_score_end : 0x7FFFFFFFFFFFFFFFLL;
    g.lat = lat ? h->lat_dev : nullptr;
    g.lat_slot = lat_slot;
    if (four) cudaStreamWaitEvent(sb, h->ev_dfree[ds], 0);   // the demap is done with these decision slots
    prof_begin(h, 5, sb);
    if (e == cudaSuccess && do_train) {
        e = launch_eq(h->ep, g, 1, h->Y[h->yw], nullptr, h->taps[h->tw], nullptr, h->dec[ds], h->winb[ds], h->winrec[ds],
                      nullptr, h->dbg_z, h->prbs, h->prbs_bits, h->st, sb);
        h->trained = 1;
    }
    if (e == cudaSuccess && g.nblk > 0) {
        if (h->cnn) {
            // learned equaliser: one segment per payload window
            long long seg_base = 2 * pay_lo - 12 - h->ybase_cur;
            e = launch_cnn_decide(rx_cnn_dev_params(h->cnn), (const float2 *)h->Y[h->yw], seg_base, s.f_k - h->ybase_cur, g.nwin, h->dec[ds],
                                  h->winb[ds], h->winrec[ds], h->prbs_bits, pay_lo, h->ep.scale, h->mq,
                                  h->dbg_z ? h->dbg_z + (pay_lo - sym_lo) : nullptr, &h->st->err, h->nsm, sb,
                                  c.cnn_bf16);
        } else {
            const float2 *zin = nullptr;
            if (c.fir_prec >= RX_FIR_BF16) {
                // frozen taps: the whole payload's filter as one tensor-core GEMM
                e = launch_fir_tc(c.fir_prec, (const float2 *)h->Y[h->yw], h->ybase_cur, pay_lo, npay,
                                  h->taps[h->tw], c.ntaps, c.eq_block, h->zbuf, &h->st->err, h->nsm, sb);
                zin = h->zbuf;
            }
            if (e == cudaSuccess)
                e = launch_eq(h->ep, g, 0, h->Y[h->yw], zin, h->taps[h->tw], h->taps[h->tw ^ 1], h->dec[ds],
                              h->winb[ds], h->winrec[ds], h->dbg_win, h->dbg_z, h->prbs, h->prbs_bits, h->st, sb);
            h->tw ^= 1;
        }
    }
    prof_end(h, 5, sb);
    // the filter slot's release is also the demap's start signal
    if (two) cudaEventRecord(h->ev_yfree[h->yw], sb);
    if (four) cudaStreamWaitEvent(st4, h->ev_yfree[h->yw], 0);
    if (e == cudaSuccess && g.nblk > 0) {
        prof_begin(h, 6, st4);
        int resolve = h->kk && !h->amb_done;
        e = launch_demap(h->ep, g, resolve, h->uw, h->dec[ds], h->winb[ds], h->winrec[ds], h->dbg_win, bits_out,
                         h->prbs_bits, h->st, st4);
        if (h->kk) h->uw ^= 1;
        h->amb_done = 1;
        prof_end(h, 6, st4);
        if (e == cudaSuccess && host_out)
            e = cudaMemcpyAsync(host_out, h->bits_stage, (size_t)((h->bps * npay + 7) / 8), cudaMemcpyDeviceToHost,
                                st4);
    }
    if (four) cudaEventRecord(h->ev_dfree[ds], st4);
    if (lat && e == cudaSuccess) h->lat_head++;
    if (h->prof_cur) h->prof_head++;
    h->prof_cur = 0;
    if (e != cudaSuccess) {
        traced(e, "rx_process enqueue");
        h->broken = 1;
        return RX_ECUDA;
    }
    h->l_e_prev = h->e_prev;
    h->l_e_k = s.e_k;
    h->l_r_prev = h->r_prev;
    h->l_r_k = s.r_k;
    h->l_f_prev = h->f_prev;
    h->l_f_k = s.f_k;
    h->l_sym_lo = sym_lo;
    h->l_pay_lo = pay_lo;
    h->l_q_k = s.q_k;
    h->l_nwin = g.nwin;
    h->l_ds = ds;
    h->e_prev = s.e_k;
    h->r_prev = s.r_k;
    h->f_prev = s.f_k;
    h->q_prev = s.q_k;
    h->calls++;
    *nbits_out = npay > 0 ? (long long)h->bps * npay : 0;
    return RX_OK;
}

rx_status rx_process(rx_handle *h, const uint8_t *in, uint8_t *bits_out, void *stream, int64_t *nbits_out)
{
    if (!h || !in || !nbits_out) return RX_EINVAL;
    if (h->broken || h->flushed) return RX_ESTATE;
    if (((uintptr_t)in) & 15) return RX_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    return enqueue_call(h, in, bits_out, nullptr, nullptr, st, st, st, nbits_out);
}

// n calls of enqueue_call on the pipeline's streams, joined onto the caller's stream
static rx_status run_batch(rx_handle *h, const uint8_t *const *ins, uint8_t *const *outs, bool host, int n,
                           void *stream, int64_t *nbits_out)
{
    cudaStream_t caller = (cudaStream_t)stream;
    const bool one = h->cfg.debug != 0;             // debug views want one call at a time
    cudaStream_t sf = one ? caller : h->front;
    cudaStream_t sb = one ? caller : h->back;
    cudaStream_t sc = one ? caller : h->copy;
    if (!one) {
        // everything earlier on the caller's stream precedes the pipeline
        if (cudaEventRecord(h->ev_fork, caller) != cudaSuccess || cudaStreamWaitEvent(sf, h->ev_fork, 0) != cudaSuccess ||
            cudaStreamWaitEvent(h->front2, h->ev_fork, 0) != cudaSuccess ||
            cudaStreamWaitEvent(h->mid, h->ev_fork, 0) != cudaSuccess ||
            cudaStreamWaitEvent(h->tail, h->ev_fork, 0) != cudaSuccess ||
            cudaStreamWaitEvent(sb, h->ev_fork, 0) != cudaSuccess || cudaStreamWaitEvent(sc, h->ev_fork, 0) != cudaSuccess)
            return RX_ECUDA;
    }
    for (int i = 0; i < n; i++) {
        cudaStream_t sm = one ? nullptr : h->mid, s4 = one ? nullptr : h->tail;
        rx_status r = host ? enqueue_call(h, nullptr, nullptr, ins[i], outs[i], sf, sb, sc, &nbits_out[i], sm, s4)
                           : enqueue_call(h, ins[i], outs[i], nullptr, nullptr, sf, sb, sc, &nbits_out[i], sm, s4);
        if (r != RX_OK) return r;
    }
    if (!one) {
        // the last demap waited for its equaliser, which waited for its matched filter
        // and field: joining the tail joins all
        if (cudaEventRecord(h->ev_join, h->tail) != cudaSuccess || cudaStreamWaitEvent(caller, h->ev_join, 0) != cudaSuccess)
            return RX_ECUDA;
    }
    return RX_OK;
}

rx_status rx_process_batch(rx_handle *h, const uint8_t *const *ins, uint8_t *const *outs, int n, void *stream,
                           int64_t *nbits_out)
{
    if (!h || !ins || !outs || !nbits_out || n <= 0) return RX_EINVAL;
    if (h->broken || h->flushed) return RX_ESTATE;
    for (int i = 0; i < n; i++)
        if (!ins[i] || (((uintptr_t)ins[i]) & 15)) return RX_EINVAL;
    return run_batch(h, ins, outs, false, n, stream, nbits_out);
}

rx_status rx_process_host_batch(rx_handle *h, const uint8_t *const *host_ins, uint8_t *const *host_outs, int n,
                                void *stream, int64_t *nbits_out)
{
    if (!h || !host_ins || !host_outs || !nbits_out || n <= 0) return RX_EINVAL;
    if (h->broken || h->flushed) return RX_ESTATE;
    for (int i = 0; i < n; i++)
        if (!host_ins[i] || !host_outs[i]) return RX_EINVAL;
    return run_batch(h, host_ins, host_outs, true, n, stream, nbits_out);
}

rx_status rx_process_host(rx_handle *h, const uint8_t *host_in, uint8_t *host_bits_out, void *stream,
                          int64_t *nbits_out)
{
    if (!h || !host_in || !host_bits_out || !nbits_out) return RX_EINVAL;
    if (h->broken || h->flushed) return RX_ESTATE;
    cudaStream_t st = (cudaStream_t)stream;
    return enqueue_call(h, nullptr, nullptr, host_in, host_bits_out, st, st, st, nbits_out);
}

rx_status rx_flush(rx_handle *h, uint8_t *bits_out, void *stream, int64_t *nbits_out)
{
    if (!h || !nbits_out) return RX_EINVAL;
    if (h->broken) return RX_ESTATE;
    *nbits_out = 0;
    if (h->flushed) return RX_OK;
    h->flushed = 1;
    if (h->calls == 0) return RX_OK;
    const rx_config &c = h->cfg;
    cudaStream_t st = (cudaStream_t)stream;
    // symbols whose centre lies inside the stream: nominal samples [0, r_end)
    const long long total = h->calls * h->nb;
    long long r_end = total;
    if (h->rs) r_end = rs_below(h, (__int128)total << 32);
    const long long S = r_end > 0 ? (r_end - 1) / h->sps + 1 : 0;
    const long long first = h->q_prev > c.ntrain ? h->q_prev : (long long)c.ntrain;
    if (S <= first) return RX_OK;
    if (!bits_out) return RX_EINVAL;
    cudaGetLastError();
    // pad: the last code repeated; the pad calls reuse the last real buffer's carrier
    // and gain (KK) or mean and deviation (PAM)
    uint8_t *pad = h->in_stage[0];
    const long long pbytes = h->nb * 3 / 2;
    const uint8_t *hend = h->kk ? h->phist[h->hw] + (long long)h->nhist * 3 / 2 : nullptr;
    const uint16_t *clast = h->kk ? nullptr : h->codes[h->cw] + h->nhist + h->nb - 1;
    k_pad_fill<<<(unsigned)((pbytes + 255) / 256 < 1024 ? (pbytes + 255) / 256 : 1024), 256, 0, st>>>(
        pad, pbytes, hend, clast, c.pack_order);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && h->kk)
        e = cudaMemcpyAsync(h->st->cg_flush, &h->st->cg[h->ew][0], 4 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        h->broken = 1;
        return RX_ECUDA;
    }
    h->flush_mode = 1;
    h->flush_par = (int)((h->calls - 1) % 3);
    h->flush_score_end = S - (c.mf_span + c.ntaps + 1) / 2;
    long long done = 0;   // bits written to bits_out
    rx_status r = RX_OK;
    for (int it = 0; h->q_prev < S && r == RX_OK && it < (1 << 20); it++) {
        int64_t nb_call = 0;
        r = enqueue_call(h, pad, h->bits_stage, nullptr, nullptr, st, st, st, &nb_call);
        if (r != RX_OK) break;
        h->pad_calls++;
        long long hi = h->l_q_k < S ? h->l_q_k : S, use = hi - h->l_pay_lo;
        if (nb_call > 0 && use > 0) {
            long long bits = (long long)h->bps * use;
            if (cudaMemcpyAsync(bits_out + done / 8, h->bits_stage, (size_t)((bits + 7) / 8), cudaMemcpyDeviceToDevice,
                                st) != cudaSuccess) {
                h->broken = 1;
                r = RX_ECUDA;
            }
            done += bits;
        }
    }
    h->flush_mode = 0;
    *nbits_out = done;
    return r;
}

rx_status rx_resampler_from_clock(double ppm, double delay, int64_t *rs_step, int64_t *rs_phase0)
{
    if (!rs_step || !rs_phase0 || !(fabs(ppm) < 9000.0) || !(fabs(delay) < 1073741824.0)) return RX_EINVAL;
    const __int128 P = (__int128)(long long)nearbyint((1.0 + ppm * 1e-6) * 4294967296.0);   // ADC period, 2^-32
    const __int128 D = (__int128)(long long)nearbyint(delay * 4294967296.0);              // delay, 2^-32
    const __int128 half = P / 2;
    const __int128 num_s = ((__int128)1 << 64) + half;
    const __int128 num_p = D * ((__int128)1 << 32) + half;
    __int128 qp = num_p / P;
    if (num_p % P != 0 && num_p < 0) qp -= 1;   // floor division
    *rs_step = (int64_t)(num_s / P);
    *rs_phase0 = (int64_t)(-qp);
    return RX_OK;
}

rx_status rx_set_fd_taps(rx_handle *h, const double *re, const double *im, int n)
{
    if (!h || !re || !h->fd || !h->fd_H || n < 1 || !(n & 1) || n > h->cfg.fd_n / 2 + 1) return RX_EINVAL;
    if (!h->kk && im)
        for (int i = 0; i < n; i++)
            if (im[i] != 0.0) return RX_EINVAL;   // the PAM filter output is taken as real
    for (int i = 0; i < n; i++)
        if (!std::isfinite(re[i]) || (im && !std::isfinite(im[i]))) return RX_EINVAL;
    const int N = h->cfg.fd_n, nbins = h->kk ? N / 2 : N;
    float2 *Hk = (float2 *)malloc(sizeof(float2) * nbins);
    if (!Hk) return RX_ENOMEM;
    fd_response(re, h->kk ? im : nullptr, n, N, h->kk, Hk);
    // calls in flight read the response: replace it only after they are done
    rx_status r = RX_OK;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(h->fd_H, Hk, sizeof(float2) * nbins, cudaMemcpyHostToDevice) != cudaSuccess)
        r = RX_ECUDA;
    free(Hk);
    if (r == RX_OK) h->cfg.fd_taps = n;
    return r;
}

rx_status rx_fd_ls_taps(const double *x_re, const double *x_im, int64_t nx, int64_t first, int step,
                        const double *a_re, const double *a_im, int64_t na, int ntaps, double ridge,
                        double *h_re, double *h_im)
{
    const bool cplx = x_im || a_im;
    if (!x_re || !a_re || !h_re || (cplx && !h_im) || ntaps < 1 || ntaps > 2049 || !(ntaps & 1) || step < 1 ||
        na < ntaps || !(ridge >= 0.0) || !std::isfinite(ridge))
        return RX_EINVAL;
    const int n = ntaps, L = (ntaps - 1) / 2;
    if (first < L || first + (int64_t)step * (na - 1) + L >= nx) return RX_EINVAL;
    typedef std::complex<double> cd;
    auto X = [&](int64_t k, int c) {   // data matrix entry: x[first + step k - (c - L)]
        const int64_t idx = first + (int64_t)step * k - c + L;
        return cd(x_re[idx], x_im ? x_im[idx] : 0.0);
    };
    std::vector<cd> R((size_t)n * n), p(n);
    // rows c1 < step directly; the others by the shift recurrence (X[k][c + step] = X[k-1][c])
    const int s0 = step < n ? step : n;
    for (int c1 = 0; c1 < s0; c1++)
        for (int c2 = 0; c2 < n; c2++) {
            cd acc = 0.0;
            for (int64_t k = 0; k < na; k++) acc += std::conj(X(k, c1)) * X(k, c2);
            R[(size_t)c1 * n + c2] = acc;
        }
    for (int c1 = s0; c1 < n; c1++)
        for (int c2 = 0; c2 < n; c2++) {
            if (c2 < s0) {
                R[(size_t)c1 * n + c2] = std::conj(R[(size_t)c2 * n + c1]);
            } else {
                const int a1 = c1 - step, a2 = c2 - step;
                R[(size_t)c1 * n + c2] = R[(size_t)a1 * n + a2] + std::conj(X(-1, a1)) * X(-1, a2) -
                                         std::conj(X(na - 1, a1)) * X(na - 1, a2);
            }
        }
    for (int c = 0; c < n; c++) {
        cd acc = 0.0;
        for (int64_t k = 0; k < na; k++) acc += std::conj(X(k, c)) * cd(a_re[k], a_im ? a_im[k] : 0.0);
        p[c] = acc;
    }
    double tr = 0.0;
    for (int c = 0; c < n; c++) tr += R[(size_t)c * n + c].real();
    for (int c = 0; c < n; c++) R[(size_t)c * n + c] += ridge * tr / n;
    // Cholesky R = G G^H (lower G in place), then G y = p and G^H h = y
    for (int j = 0; j < n; j++) {
        double d = R[(size_t)j * n + j].real();
        for (int q = 0; q < j; q++) d -= std::norm(R[(size_t)j * n + q]);
        if (!(d > 0.0)) return RX_EINVAL;
        const double gjj = std::sqrt(d);
        R[(size_t)j * n + j] = gjj;
        for (int i = j + 1; i < n; i++) {
            cd v = R[(size_t)i * n + j];
            for (int q = 0; q < j; q++) v -= R[(size_t)i * n + q] * std::conj(R[(size_t)j * n + q]);
            R[(size_t)i * n + j] = v / gjj;
        }
    }
    std::vector<cd> y(n);
    for (int i = 0; i < n; i++) {
        cd v = p[i];
        for (int q = 0; q < i; q++) v -= R[(size_t)i * n + q] * y[q];
        y[i] = v / R[(size_t)i * n + i].real();
    }
    for (int i = n - 1; i >= 0; i--) {
        cd v = y[i];
        for (int q = i + 1; q < n; q++) v -= std::conj(R[(size_t)q * n + i]) * p[q];
        p[i] = v / R[(size_t)i * n + i].real();   // p now holds h
    }
    for (int c = 0; c < n; c++) {
        h_re[c] = p[c].real();
        if (h_im) h_im[c] = cplx ? p[c].imag() : 0.0;
    }
    return RX_OK;
}

static double q_from_ber(double ber)
{
    if (!(ber > 0)) return INFINITY;
    if (ber >= 0.5) return -INFINITY;
    double lo = 0, hi = 30, t = 2 * ber;
    for (int i = 0; i < 200; i++) {
        double m = 0.5 * (lo + hi);
        if (erfc(m) > t) lo = m;
        else hi = m;
    }
    return 20.0 * log10(sqrt(2.0) * 0.5 * (lo + hi));
}

rx_status rx_stats(rx_handle *h, rx_stats_t *o, void *stream)
{
    if (!h || !o) return RX_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return RX_ECUDA;
    DevState s;
    if (cudaMemcpy(&s, h->st, sizeof s, cudaMemcpyDeviceToHost) != cudaSuccess) return RX_ECUDA;
    memset(o, 0, sizeof *o);
    o->calls = h->calls - h->pad_calls;
    o->samples = o->calls * h->nb;
    o->symbols = (int64_t)s.cnt[C_SYMBOLS];
    o->bits = (int64_t)s.cnt[C_BITS];
    o->bit_errors = (int64_t)s.cnt[C_BITERR];
    o->raw_bit_errors = (int64_t)s.cnt[C_RAWERR];
    o->sym_errors = (int64_t)s.cnt[C_SYMERR];
    o->slip_windows = (int64_t)s.cnt[C_SLIP];
    o->near_threshold = (int64_t)s.cnt[C_NEAR];
    o->ambiguous_windows = (int64_t)s.cnt[C_AMBIG];
    o->windows = (int64_t)s.cnt[C_WINDOWS];
    o->amb_rot = s.amb_r;
    o->device_error = s.err;
    o->ber = o->bits ? (double)o->bit_errors / (double)o->bits : 0.0;
    o->q_db = q_from_ber(o->ber);
    if (h->lat_dev) {
        unsigned long long cnt[3];   // n, miss, max_ns
        if (launch_lat_flush(h->lat_dev, (cudaStream_t)stream) != cudaSuccess ||
            cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess || cudaMemcpy(cnt, &h->lat_dev->n, sizeof cnt, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(h->lat_hist, h->lat_dev->hist, sizeof(uint32_t) * kLatBins, cudaMemcpyDeviceToHost) !=
                cudaSuccess)
            return RX_ECUDA;
        const double max_ms = (double)cnt[2] * 1e-6;
        o->lat_calls = (int64_t)cnt[0];
        o->deadline_misses = (int64_t)cnt[1];
        o->deadline_ms = h->lat_budget;
        o->lat_p50_ms = lat_pct(h->lat_hist, (long long)cnt[0], max_ms, 0.50);
        o->lat_p99_ms = lat_pct(h->lat_hist, (long long)cnt[0], max_ms, 0.99);
        o->lat_max_ms = max_ms;
    }
    return RX_OK;
}

rx_status rx_clock_estimate(rx_handle *h, double *ppm, double *delay, void *stream)
{
    if (!h || !ppm || !delay) return RX_EINVAL;
    if (!h->clk) return RX_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return RX_ECUDA;
    // outputs per block at 2 samples/symbol: N/4 (KK, 4 -> 2 sps) or N/2 (PAM)
    const long long N = h->cfg.fd_n, per = h->kk ? N / 4 : N / 2;
    const long long b0 = h->l_f_prev / per, n = (h->l_f_k - h->l_f_prev) / per;
    if (n < 2) return RX_ESTATE;
    float2 *c = (float2 *)malloc(sizeof(float2) * n);
    if (!c) return RX_ENOMEM;
    if (cudaMemcpy(c, h->clk, sizeof(float2) * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
        free(c);
        return RX_ECUDA;
    }
    // d_b = -(P / 2 pi) arg C_b unwrapped (period P = samples per symbol: 4 KK, 2 PAM),
    // least-squares d_b = -tau0 - eps centre_b, centre_b = (N/2) b + N/4 (the middle of
    // block b's inputs)
    const double pi = 3.14159265358979323846;
    const double P = h->kk ? 4.0 : 2.0, Hp = 0.5 * P;
    const double x0 = (double)((N / 2) * b0 + N / 4);
    double prev = 0, off = 0, sx = 0, sy = 0, sxx = 0, sxy = 0;
    for (long long i = 0; i < n; i++) {
        double d = -P / (2.0 * pi) * atan2((double)c[i].y, (double)c[i].x);
        if (i > 0) {
            while (d + off - prev > Hp) off -= P;
            while (d + off - prev < -Hp) off += P;
        }
        const double y = d + off, x = (double)(N / 2) * (double)i;
        prev = y;
        sx += x;
        sy += y;
        sxx += x * x;
        sxy += x * y;
    }
    free(c);
    const double nb = (double)n, slope = (nb * sxy - sx * sy) / (nb * sxx - sx * sx);
    double tau0 = -((sy - slope * sx) / nb - slope * x0);
    while (tau0 > Hp) tau0 -= P;
    while (tau0 <= -Hp) tau0 += P;
    *ppm = -slope * 1e6;
    *delay = tau0;
    return RX_OK;
}

// the tracker state after everything enqueued on the stream
static rx_status read_track(rx_handle *h, void *stream, ClockTrack *ck)
{
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return RX_ECUDA;
    if (cudaMemcpy(ck, &h->st->ck, sizeof *ck, cudaMemcpyDeviceToHost) != cudaSuccess) return RX_ECUDA;
    return RX_OK;
}

rx_status rx_clock_track(rx_handle *h, double *ppm, double *delay, int64_t *nblocks, void *stream)
{
    if (!h || !ppm || !delay || !h->cfg.clk_track) return RX_EINVAL;
    ClockTrack ck;
    rx_status r = read_track(h, stream, &ck);
    if (r != RX_OK) return r;
    if (nblocks) *nblocks = ck.n;
    if (ck.n < 2) return RX_ESTATE;
    // the line d = -delay - 1e-6 ppm c over the block centres c, delay at stream index 0
    const double P = (double)h->sps, Hp = 0.5 * P, n = (double)ck.n;
    const double slope = (n * ck.sxy - ck.sx * ck.sy) / (n * ck.sxx - ck.sx * ck.sx);
    double tau0 = -((ck.sy - slope * ck.sx) / n - slope * ck.x0);
    while (tau0 > Hp) tau0 -= P;
    while (tau0 <= -Hp) tau0 += P;
    *ppm = -slope * 1e6;
    *delay = tau0;
    return RX_OK;
}

// new piece of the resampler accumulator from the next nominal sample on, and a
// restart of the clock tracker
static rx_status apply_resampler(rx_handle *h, long long step, long long nudge, cudaStream_t st)
{
    if (step < 4252017623LL || step > 4337916969LL) return RX_EBOUNDS;
    h->rs_psi0 = rs_psi(h, h->r_prev) + (__int128)nudge;
    h->rs_r0 = h->r_prev;
    h->cfg.rs_step = step;
    if (cudaMemsetAsync(&h->st->ck, 0, sizeof(ClockTrack), st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RX_ECUDA;
    return RX_OK;
}

rx_status rx_set_resampler(rx_handle *h, int64_t step, int64_t nudge, void *stream)
{
    if (!h || !h->rs || nudge <= -(1LL << 36) || nudge >= (1LL << 36)) return RX_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return RX_ECUDA;
    rx_status r = apply_resampler(h, step, nudge, (cudaStream_t)stream);
    return r == RX_EBOUNDS ? RX_EINVAL : r;
}

rx_status rx_clock_retime(rx_handle *h, int64_t *step_out, int64_t *nudge_out, void *stream)
{
    if (!h || !h->rs || !h->cfg.clk_track) return RX_EINVAL;
    ClockTrack ck;
    rx_status r = read_track(h, stream, &ck);
    if (r != RX_OK) return r;
    if (ck.n < 2) return RX_ESTATE;
    // line y = y0 + s x of the unwrapped delays (x relative to the first block's centre)
    const double P = (double)h->sps, Hp = 0.5 * P, n = (double)ck.n;
    const double s = (n * ck.sxy - ck.sx * ck.sy) / (n * ck.sxx - ck.sx * ck.sx);
    const double y0 = (ck.sy - s * ck.sx) / n;
    double w = y0 + s * ((double)h->r_prev - ck.x0);
    w -= P * floor(w / P);
    if (w > Hp) w -= P;
    const long long step = llround((double)h->cfg.rs_step * (1.0 + s));
    const long long nudge = llround(w * (double)h->cfg.rs_step);
    r = apply_resampler(h, step, nudge, (cudaStream_t)stream);
    if (r != RX_OK) return r;
    if (step_out) *step_out = step;
    if (nudge_out) *nudge_out = nudge;
    return RX_OK;
}

rx_status rx_debug_copy(rx_handle *h, int what, void *dst, int64_t cap, int64_t *count, int64_t *start, void *stream)
{
    if (!h || !count || !start) return RX_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return RX_ECUDA;
    const void *src = nullptr;
    long long n = 0, s0 = 0;
    size_t el = 0;
    switch (what) {
    case RX_DBG_FIELD:
        if (!h->kk) return RX_EINVAL;
        n = h->l_e_k - h->l_e_prev;
        s0 = h->l_e_prev;
        src = h->E[h->ew] + kEHist;
        el = sizeof(float2);
        break;
    case RX_DBG_RS:
        if (!h->rs) return RX_EINVAL;
        n = h->l_r_k - h->l_r_prev;
        s0 = h->l_r_prev;
        src = h->R[h->rw] + (h->l_r_prev - h->rbase_cur);
        el = sizeof(float2);
        break;
    case RX_DBG_CLK:
        if (!h->clk) return RX_EINVAL;
        n = (h->l_f_k - h->l_f_prev) / (h->kk ? h->cfg.fd_n / 4 : h->cfg.fd_n / 2);
        s0 = h->l_f_prev / (h->kk ? h->cfg.fd_n / 4 : h->cfg.fd_n / 2);
        src = h->clk;
        el = sizeof(float2);
        break;
    case RX_DBG_MF:
        n = h->l_f_k - h->l_f_prev;
        s0 = h->l_f_prev;
        el = h->kk ? sizeof(float2) : sizeof(float);
        src = (const char *)h->Y[h->yw] + (size_t)(h->l_f_prev - h->ybase_cur) * el;
        break;
    case RX_DBG_SOFT:
        if (!h->dbg_z) return RX_EINVAL;
        n = h->l_q_k - h->l_sym_lo;
        s0 = h->l_sym_lo;
        src = h->dbg_z;
        el = sizeof(float2);
        break;
    case RX_DBG_DEC:
        n = h->l_q_k - h->l_pay_lo;
        if (n < 0) n = 0;
        s0 = h->l_pay_lo;
        src = h->dec[h->l_ds];
        el = 1;
        break;
    case RX_DBG_WIN:
        if (!h->dbg_win) return RX_EINVAL;
        n = h->l_nwin;
        s0 = 0;
        src = h->dbg_win;
        el = sizeof(float4);
        break;
    case RX_DBG_TAPS:
        n = h->cfg.ntaps;
        s0 = 0;
        src = h->taps[h->tw];
        el = sizeof(float2);
        break;
    case RX_DBG_CODES:
        n = h->nb;
        s0 = (h->calls - 1) * h->nb;
        src = h->codes[h->cw] + h->nhist;
        el = sizeof(uint16_t);
        break;
    case RX_DBG_SCAL: {
        DevState s;
        if (cudaMemcpy(&s, h->st, sizeof s, cudaMemcpyDeviceToHost) != cudaSuccess) return RX_ECUDA;
        double v[5] = {s.cg[h->ew][0], s.cg[h->ew][1], s.cg[h->ew][2], s.pam_mu, s.pam_inv_sd};
        *count = 5;
        *start = 0;
        if (dst) memcpy(dst, v, sizeof(double) * (size_t)(cap < 5 ? cap : 5));
        return RX_OK;
    }
    default:
        return RX_EINVAL;
    }
    *count = n;
    *start = s0;
    if (dst && cap > 0 && n > 0) {
        long long m = n < cap ? n : cap;
        if (cudaMemcpy(dst, src, (size_t)m * el, cudaMemcpyDeviceToHost) != cudaSuccess) return RX_ECUDA;
    }
    return RX_OK;
}

rx_status rx_profile(rx_handle *h, int enable)
{
    if (!h || enable < 0) return RX_EINVAL;
    if (enable && !h->prof_ev) {
        h->prof_ev = (cudaEvent_t *)calloc((size_t)kProfRing * kEvPerCall, sizeof(cudaEvent_t));
        h->prof_used = (int *)calloc(kProfRing, sizeof(int));
        if (!h->prof_ev || !h->prof_used) return RX_ENOMEM;
        for (int i = 0; i < kProfRing * kEvPerCall; i++)
            if (cudaEventCreate(&h->prof_ev[i]) != cudaSuccess) return RX_ECUDA;
    }
    h->prof_on = enable;
    return RX_OK;
}

rx_status rx_profile_read(rx_handle *h, double *ms, int n, int64_t *calls)
{
    if (!h || !ms || !calls || n < 0 || n > kStages) return RX_EINVAL;
    while (h->prof_tail < h->prof_head) prof_harvest_one(h);
    for (int i = 0; i < n; i++) ms[i] = h->prof_ms[i];
    *calls = h->prof_calls;
    memset(h->prof_ms, 0, sizeof h->prof_ms);
    h->prof_calls = 0;
    return RX_OK;
}

rx_status rx_fir_block(const float *y, int64_t ny, const float *w, int ntaps, int prec, int64_t nsym,
                       int scale_block, float *z_out, int32_t *status, void *stream)
{
    if (!y || !w || !z_out || !status || ntaps < 1 || ntaps > kMaxTaps || !(ntaps & 1) || nsym <= 0 ||
        nsym % 16 || prec < RX_FIR_BF16 || prec > RX_FIR_FP8 || scale_block < 16 || scale_block % 16 ||
        2048 % scale_block || nsym % scale_block || ny < 2 * nsym + ntaps + 1 || (((uintptr_t)y) & 15) ||
        (((uintptr_t)z_out) & 15))
        return RX_EINVAL;
    // y[j] holds stream index j - TH, so z_k = sum_i conj(w_i) y[2k + TH - i] in stream terms
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        prepare_fir_tc(prec) != cudaSuccess)
        return RX_ECUDA;
    cudaError_t e = launch_fir_tc(prec, (const float2 *)y, -(long long)((ntaps - 1) / 2), 0, nsym,
                                  (const float2 *)w, ntaps, scale_block, (float2 *)z_out, (int *)status, nsm,
                                  (cudaStream_t)stream);
    return e == cudaSuccess ? RX_OK : RX_ECUDA;
}

// ----------------------------------------------------------------- groups
// Members run on worker streams forked from the caller's stream; member i goes
// to worker i mod nw in order of decreasing buffer length.  With RX_GROUP_GRAPH
// each round is captured into a CUDA graph whose executable instance is
// updated in place (the topology repeats round to round; only kernel
// parameters change) and launched once.
struct rx_group {
    int n, nw, flags;
    rx_handle **m;
    int *order;
    cudaStream_t ws[8];
    cudaEvent_t fork, done[8];
    cudaGraphExec_t exec;
    int *tuned;   // per member: kk_front | eq_warps << 4
};

__global__ void k_fill_bytes(uint8_t *p, long long n, unsigned seed)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        unsigned x = (unsigned)i * 2654435761u ^ seed;
        x ^= x >> 15;
        x *= 2246822519u;
        x ^= x >> 13;
        p[i] = (uint8_t)x;
    }
}

// time `calls` calls of a fresh handle of this shape and implementation choice
static float time_variant(int fmt, double baud, double fs, long long nb, rx_config c, const uint8_t *const *bufs,
                          int nbuf, uint8_t *bits, cudaStream_t st)
{
    rx_handle *t = nullptr;
    rx_status cr = rx_create((rx_format)fmt, baud, fs, nb, &c, &t);
    if (cr != RX_OK) {
        if (trace_on()) fprintf(stderr, "rx: tuner candidate rejected by rx_create: %s\n", rx_strerror(cr));
        cudaGetLastError();
        return -1.f;
    }
    float best = -1.f;
    int64_t nbits;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    bool ok = true;
    for (int i = 0; i < 4 && ok; i++) ok = rx_process(t, bufs[i % nbuf], bits, st, &nbits) == RX_OK;   // training
    for (int rep = 0; rep < 3 && ok; rep++) {
        cudaEventRecord(a, st);
        for (int i = 0; i < 3 && ok; i++) ok = rx_process(t, bufs[i % nbuf], bits, st, &nbits) == RX_OK;
        cudaEventRecord(b, st);
        float ms = 0.f;
        if (ok && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
            best = (best < 0.f || ms < best) ? ms : best;
    }
    cudaStreamSynchronize(st);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    rx_destroy(t);
    cudaError_t e = cudaGetLastError();   // a failed candidate leaves nothing behind
    if (!ok || e != cudaSuccess) traced(e != cudaSuccess ? e : cudaErrorUnknown, "tuner candidate");
    return ok ? best : -1.f;
}

// pick the fastest implementation choice (front-end kernel structure, equaliser
// CTA shape) for each distinct member shape, on pseudo-random input
static rx_status tune_group(rx_group *g)
{
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return RX_ECUDA;
    rx_status r = RX_OK;
    for (int i = 0; i < g->n && r == RX_OK; i++) {
        rx_handle *h = g->m[i];
        int j = 0;   // an earlier member of the same shape
        for (; j < i; j++) {
            rx_handle *o = g->m[j];
            if (o->fmt == h->fmt && o->nb == h->nb && o->sps == h->sps && !memcmp(&o->cfg, &h->cfg, sizeof h->cfg))
                break;
        }
        if (j < i) {
            g->tuned[i] = g->tuned[j];
        } else {
            const int nbuf = 2;
            uint8_t *bufs[nbuf] = {nullptr, nullptr}, *bits = nullptr;
            size_t bytes = (size_t)(h->nb * 3 / 2);
            bool ok = cudaMalloc(&bits, (size_t)(rx_max_bits(h) / 8 + 16)) == cudaSuccess;
            for (int b = 0; b < nbuf && ok; b++) {
                ok = cudaMalloc(&bufs[b], bytes + 16) == cudaSuccess;
                if (ok) k_fill_bytes<<<(unsigned)((bytes + 255) / 256), 256, 0, st>>>(bufs[b], (long long)bytes, 977u * (b + 1));
            }
            float best = -1.f;
            int pick = h->cfg.kk_front | (h->ep.warps << 4);
            int fronts = (h->kk && h->N == 65536) ? 2 : 1;
            const int warps[3] = {2, 4, 8};
            double baud = 4e9 / h->sps;
            for (int f = 0; f < fronts && ok; f++)
                for (int w = 0; w < 3 && ok; w++) {
                    rx_config c = h->cfg;
                    c.kk_front = f;
                    c.eq_warps = warps[w];
                    c.debug = 0;
                    float ms = time_variant(h->fmt, baud, 4e9, h->nb, c, bufs, nbuf, bits, st);
                    if (ms > 0.f && (best < 0.f || ms < best)) {
                        best = ms;
                        pick = f | (warps[w] << 4);
                    }
                }
            for (int b = 0; b < nbuf; b++) cudaFree(bufs[b]);
            cudaFree(bits);
            if (!ok) r = RX_ECUDA;
            g->tuned[i] = pick;
        }
        // apply: neither choice changes the stream state
        h->cfg.kk_front = g->tuned[i] & 15;
        h->cfg.eq_warps = g->tuned[i] >> 4;
        h->ep.warps = h->cfg.eq_warps;
        if (prepare_eq(h->ep) != cudaSuccess) r = RX_ECUDA;
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return r;
}

rx_status rx_group_destroy(rx_group *g)
{
    if (!g) return RX_EINVAL;
    for (int w = 0; w < g->nw; w++) {
        if (g->ws[w]) {
            cudaStreamSynchronize(g->ws[w]);
            cudaStreamDestroy(g->ws[w]);
        }
        if (g->done[w]) cudaEventDestroy(g->done[w]);
    }
    if (g->fork) cudaEventDestroy(g->fork);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    free(g->m);
    free(g->order);
    free(g->tuned);
    free(g);
    return RX_OK;
}

rx_status rx_group_create(rx_handle *const *members, int n, int flags, rx_group **out)
{
    if (!members || !out || n < 1 || (flags & ~(RX_GROUP_GRAPH | RX_GROUP_TUNE))) return RX_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; i++) {
        if (!members[i] || members[i]->broken || members[i]->flushed) return RX_EINVAL;
        for (int j = 0; j < i; j++)
            if (members[j] == members[i]) return RX_EINVAL;
    }
    rx_group *g = (rx_group *)calloc(1, sizeof(rx_group));
    if (!g) return RX_ENOMEM;
    g->n = n;
    g->flags = flags;
    g->nw = n < 8 ? n : 8;
    g->m = (rx_handle **)malloc(sizeof(rx_handle *) * n);
    g->order = (int *)malloc(sizeof(int) * n);
    g->tuned = (int *)calloc(n, sizeof(int));
    if (!g->m || !g->order || !g->tuned) {
        rx_group_destroy(g);
        return RX_ENOMEM;
    }
    for (int i = 0; i < n; i++) {
        g->m[i] = members[i];
        g->order[i] = i;
        g->tuned[i] = members[i]->cfg.kk_front | (members[i]->ep.warps << 4);
    }
    // longest buffers first, dealt round-robin over the workers
    for (int i = 1; i < n; i++)
        for (int j = i; j > 0 && g->m[g->order[j]]->nb > g->m[g->order[j - 1]]->nb; j--) {
            int t = g->order[j];
            g->order[j] = g->order[j - 1];
            g->order[j - 1] = t;
        }
    bool ok = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int w = 0; w < g->nw && ok; w++)
        ok = cudaStreamCreateWithFlags(&g->ws[w], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&g->done[w], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        rx_group_destroy(g);
        return RX_ECUDA;
    }
    if (flags & RX_GROUP_TUNE) {
        rx_status r = tune_group(g);
        if (r != RX_OK) {
            rx_group_destroy(g);
            return r;
        }
    }
    *out = g;
    return RX_OK;
}

rx_status rx_group_tuning(const rx_group *g, int i, int32_t *kk_front, int32_t *eq_warps)
{
    if (!g || i < 0 || i >= g->n || !kk_front || !eq_warps) return RX_EINVAL;
    *kk_front = g->tuned[i] & 15;
    *eq_warps = g->tuned[i] >> 4;
    return RX_OK;
}

rx_status rx_group_process(rx_group *g, const uint8_t *const *ins, uint8_t *const *outs, void *stream,
                           int64_t *nbits_out)
{
    if (!g || !ins || !outs || !nbits_out) return RX_EINVAL;
    cudaStream_t caller = (cudaStream_t)stream;
    const bool graph = (g->flags & RX_GROUP_GRAPH) != 0;
    if (graph && !caller) return RX_EINVAL;   // the legacy default stream cannot be captured
    for (int i = 0; i < g->n; i++) {
        if (g->m[i]->broken || g->m[i]->flushed) return RX_ESTATE;
        if (!ins[i] || (((uintptr_t)ins[i]) & 15)) return RX_EINVAL;
    }
    if (graph && cudaStreamBeginCapture(caller, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return RX_ECUDA;
    cudaError_t e = cudaEventRecord(g->fork, caller);
    for (int w = 0; w < g->nw && e == cudaSuccess; w++) e = cudaStreamWaitEvent(g->ws[w], g->fork, 0);
    rx_status r = e == cudaSuccess ? RX_OK : RX_ECUDA;
    for (int k = 0; k < g->n && r == RX_OK; k++) {
        int i = g->order[k];
        rx_handle *h = g->m[i];
        cudaStream_t ws = g->ws[k % g->nw];
        int prof = h->prof_on;
        h->prof_on = 0;   // no stage or latency events inside a group round
        h->in_group = 1;
        r = enqueue_call(h, ins[i], outs[i], nullptr, nullptr, ws, ws, ws, &nbits_out[i]);
        h->in_group = 0;
        h->prof_on = prof;
    }
    for (int w = 0; w < g->nw && r == RX_OK; w++)
        if (cudaEventRecord(g->done[w], g->ws[w]) != cudaSuccess || cudaStreamWaitEvent(caller, g->done[w], 0) != cudaSuccess)
            r = RX_ECUDA;
    if (!graph) return r;
    cudaGraph_t gr = nullptr;
    cudaError_t ec = cudaStreamEndCapture(caller, &gr);
    if (r != RX_OK || ec != cudaSuccess || !gr) {
        // the members' stream positions advanced for work that never ran
        for (int i = 0; i < g->n; i++) g->m[i]->broken = 1;
        if (gr) cudaGraphDestroy(gr);
        cudaGetLastError();
        return r != RX_OK ? r : RX_ECUDA;
    }
    if (g->exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(g->exec, gr, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(g->exec);
            g->exec = nullptr;
        }
    }
    if (!g->exec) ec = cudaGraphInstantiate(&g->exec, gr, 0);
    if (ec == cudaSuccess) ec = cudaGraphLaunch(g->exec, caller);
    cudaGraphDestroy(gr);
    if (ec != cudaSuccess) {
        for (int i = 0; i < g->n; i++) g->m[i]->broken = 1;
        return RX_ECUDA;
    }
    return RX_OK;
}

rx_status rx_set_cnn(rx_handle *h, const rx_cnn *cnn)
{
    if (!h || (cnn && !h->kk)) return RX_EINVAL;
    if (cnn && prepare_cnn_rx() != cudaSuccess) return RX_ECUDA;
    h->cnn = cnn;
    return RX_OK;
}

rx_status rx_set_taps(rx_handle *h, const double *re, const double *im, int n)
{
    if (!h || !re || n < 0 || n > h->cfg.ntaps) return RX_EINVAL;
    float2 t[32];
    if (cudaMemcpy(t, h->taps[h->tw], sizeof t, cudaMemcpyDeviceToHost) != cudaSuccess) return RX_ECUDA;
    for (int i = 0; i < n; i++) t[i] = make_float2((float)re[i], im ? (float)im[i] : 0.f);
    if (cudaMemcpy(h->taps[h->tw], t, sizeof t, cudaMemcpyHostToDevice) != cudaSuccess) return RX_ECUDA;
    return RX_OK;
}

}  // extern "C"
