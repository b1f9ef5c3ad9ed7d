// C ABI of the receiver library: handle lifetime, per-call scheduling of the
// kernels, constant tables, statistics and debug copies.  See include/rx.h.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "rx_internal.cuh"

using namespace rxk;

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
    uint8_t *phist[2];              // KK: packed history, ping-pong
    int hw;
    float2 *fftws, *E[2];
    void *Y[2];
    CarrierPartial *partials;
    uint8_t *dec, *winb, *prbs;
    uint32_t *prbs_bits;            // the PRBS period bit-packed MSB first, first 256 bits repeated
    uint4 *winrec;                  // per payload window: errors under the four rotations, near count
    float2 *taps[2], *twN, *twN2, *ds_tab;
    float *lnt, *sqt;
    float *rrc;
    float rrc_host[2 * 64 + 1];     // host copy of the matched-filter taps
    float4 *dbg_win;
    float2 *dbg_z;
    DevState *st;
    uint8_t *in_stage, *bits_stage;
    long long dec_cap, win_cap, y_cap;
    // stage timing: a ring of event sets, one per profiled call
    const rx_cnn *cnn;              // learned equaliser for the payload, or null
    int prof_on;
    cudaEvent_t *prof_ev;      // kProfRing * kStages1 events
    int *prof_used;            // stages recorded in each ring slot (bitmask of boundaries)
    long long prof_head, prof_tail;
    double prof_ms[8];
    long long prof_calls;
};

static const int kProfRing = 1024;
static const int kStages = 7;        // unpack, kk_fwd, kk_rows, kk_inv, mf, eq, demap
static const int kStages1 = kStages + 1;

// record the boundary before stage `stage` (kStages = end of call)
static void prof_mark(rx_handle *h, int stage, cudaStream_t st)
{
    if (!h->prof_on) return;
    long long slot = h->prof_head % kProfRing;
    cudaEventRecord(h->prof_ev[slot * kStages1 + stage], st);
    h->prof_used[slot] |= 1 << stage;
}

void rxk::prof_stage(void *prof, int stage, cudaStream_t st)
{
    if (prof) prof_mark((rx_handle *)prof, stage, st);
}

// harvest the oldest recorded call (blocking on its last event)
static void prof_harvest_one(rx_handle *h)
{
    long long slot = h->prof_tail % kProfRing;
    int used = h->prof_used[slot];
    cudaEvent_t *ev = h->prof_ev + slot * kStages1;
    cudaEventSynchronize(ev[kStages]);
    for (int s = 0; s < kStages; s++) {
        if (!(used & (1 << s))) continue;
        int e = s + 1;
        while (e < kStages && !(used & (1 << e))) e++;   // next recorded boundary
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[s], ev[e]) == cudaSuccess) h->prof_ms[s] += ms;
    }
    h->prof_used[slot] = 0;
    h->prof_tail++;
    h->prof_calls++;
}

// ---------------------------------------------------------------- host tables
// Root-raised cosine, sps*span+1 taps, unit energy, zero phase (textbook form).
static void rrc_taps(double beta, int sps, int span, double *h)
{
    const double pi = 3.14159265358979323846;
    int half = sps * span / 2, n = 2 * half + 1;
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
    long long avail, e_k, f_k, s_k, q_k;
};
static Sched schedule(const rx_handle *h, long long calls, long long q_prev)
{
    Sched s;
    s.avail = (calls + 1) * h->nb;
    s.e_k = h->kk ? s.avail - h->V / 2 : s.avail;
    if (s.e_k < 0) s.e_k = 0;
    s.f_k = (s.e_k >= h->hmf + 1) ? (s.e_k - h->hmf - 1) / h->decim + 1 : 0;
    s.s_k = (s.f_k >= h->th + 1) ? (s.f_k - h->th - 1) / 2 + 1 : 0;
    long long nt = h->cfg.ntrain, B = h->cfg.eq_block;
    s.q_k = (s.s_k >= nt) ? nt + ((s.s_k - nt) / B) * B : 0;
    if (s.q_k < q_prev) s.q_k = q_prev;
    return s;
}

extern "C" {

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
    c->eq_block = 256;
    c->win = 64;
    c->mu = 1e-3;
    c->mu_train = 1e-3;
    c->mu_cma = 1e-3;
    c->bps_b = 32;
    c->amb_syms = kk ? 1024 : 0;
    c->prbs_seed = 1;
    c->debug = 0;
    return RX_OK;
}

int64_t rx_max_bits(const rx_handle *h)
{
    if (!h) return 0;
    return (long long)h->bps * (h->nb / h->sps + h->cfg.eq_block + h->cfg.ntrain + 64);
}

void rx_destroy(rx_handle *h)
{
    if (!h) return;
    void *ptrs[] = {h->codes[0], h->codes[1], h->fftws, h->E[0], h->E[1], h->Y[0], h->Y[1], h->partials,
                    h->dec, h->winb, h->prbs, h->taps[0], h->taps[1], h->twN, h->twN2, h->ds_tab,
                    h->rrc, h->dbg_win, h->dbg_z, h->st, h->in_stage, h->bits_stage, h->lnt, h->sqt,
                    h->prbs_bits, h->winrec, h->phist[0], h->phist[1]};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->prof_ev) {
        for (int i = 0; i < kProfRing * kStages1; i++) cudaEventDestroy(h->prof_ev[i]);
        free(h->prof_ev);
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
    if (c.pack_order < 0 || c.pack_order > 1 || c.ntaps < 1 || c.ntaps > kMaxTaps || !(c.ntaps & 1) ||
        c.win != kWin || c.eq_block < kWin || c.eq_block % kWin || c.ntrain < 0 || c.ntrain % kWin ||
        c.mf_span < 0 || c.mf_span % 2 || sps * c.mf_span / 2 > kEHist / 2 || !(c.rrc_beta >= 0) ||
        c.rrc_beta > 1 || c.eq_block > 4096)
        return RX_EINVAL;
    if (kk && (c.ncma < 0 || c.ncma > c.ntrain || c.ncma % kWin || c.bps_b < 1 || c.bps_b > 32 ||
               c.ds_den < 1 || c.ds_num < 0 || c.amb_syms < 0 || c.amb_syms % kWin || c.amb_syms > 4096 ||
               !(c.ols_n == 4096 || c.ols_n == 65536) || c.ols_v < 64 || c.ols_v % 64 || c.ols_v >= c.ols_n))
        return RX_EINVAL;
    rx_handle *h = (rx_handle *)calloc(1, sizeof(rx_handle));
    if (!h) return RX_ENOMEM;
    h->fmt = f;
    h->kk = kk;
    h->bps = (f == RX_PAM2) ? 1 : (f == RX_PAM4) ? 2 : (f == RX_PAM8) ? 3 : (f == RX_KK_QPSK) ? 2 : 4;
    h->mq = kk ? ((f == RX_KK_QPSK) ? 2 : 4) : (1 << h->bps);
    h->sps = sps;
    h->decim = sps / 2;
    h->hmf = sps * c.mf_span / 2;
    h->th = (c.ntaps - 1) / 2;
    h->nb = buf_len;
    h->cfg = c;
    h->nhist = kk ? c.ols_n : kPamHist;
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

    long long nb = buf_len;
    long long symcap = nb / sps + 2LL * c.eq_block + c.ntrain + 256;
    h->dec_cap = symcap;
    h->win_cap = symcap / kWin + 1;
    h->y_cap = nb / h->decim + 2LL * c.eq_block + 2LL * c.ntrain + 256;
    size_t yel = kk ? sizeof(float2) : sizeof(float);
    for (int i = 0; i < 2; i++) {
        RX_ALLOC(h->codes[i], (h->nhist + nb) * sizeof(uint16_t));
        RX_ALLOC(h->Y[i], h->y_cap * yel);
        RX_ALLOC(h->taps[i], 32 * sizeof(float2));
    }
    if (kk) {
        for (int i = 0; i < 2; i++) RX_ALLOC(h->E[i], (kEHist + nb) * sizeof(float2));
        for (int i = 0; i < 2; i++) RX_ALLOC(h->phist[i], (size_t)h->nhist * 3 / 2 + 16);
        RX_ALLOC(h->fftws, (size_t)h->npairs_max * h->N * sizeof(float2));
        int gx = (h->N2 + kCtaK1 - 1) / kCtaK1;
        RX_ALLOC(h->partials, (size_t)gx * h->npairs_max * sizeof(CarrierPartial));
        RX_ALLOC(h->twN, kk_tw_entries(h->N) * sizeof(float2));
        RX_ALLOC(h->twN2, kk_tw_entries(h->N2) * sizeof(float2));
        RX_ALLOC(h->lnt, kLutCodes * sizeof(float));
        RX_ALLOC(h->sqt, kLutCodes * sizeof(float));
        RX_ALLOC(h->ds_tab, c.ds_den * sizeof(float2));
    }
    RX_ALLOC(h->dec, h->dec_cap);
    RX_ALLOC(h->winb, h->win_cap);
    RX_ALLOC(h->prbs, 32767 + 256);
    RX_ALLOC(h->prbs_bits, 1040 * sizeof(uint32_t));
    RX_ALLOC(h->winrec, h->win_cap * sizeof(uint4));
    RX_ALLOC(h->rrc, (2 * h->hmf + 1) * sizeof(float));
    RX_ALLOC(h->st, sizeof(DevState));
    RX_ALLOC(h->in_stage, nb * 3 / 2 + 16);
    RX_ALLOC(h->bits_stage, rx_max_bits(h) / 8 + 16);
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
    uint32_t pw[1040];
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
        float *ln = (float *)malloc(sizeof(float) * kLutCodes), *sq = (float *)malloc(sizeof(float) * kLutCodes);
        kk_host_tables(h->N, ln, sq, t1, t2);
        e = cudaMemcpy(h->twN, t1, sizeof(float2) * n1, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->twN2, t2, sizeof(float2) * n2, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->lnt, ln, sizeof(float) * kLutCodes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->sqt, sq, sizeof(float) * kLutCodes, cudaMemcpyHostToDevice);
        free(t1);
        free(t2);
        free(ln);
        free(sq);
        float2 *ds = (float2 *)malloc(sizeof(float2) * c.ds_den);
        twiddles(c.ds_den, ds);      // e^{-2 pi i p / den}
        if (e == cudaSuccess) e = cudaMemcpy(h->ds_tab, ds, sizeof(float2) * c.ds_den, cudaMemcpyHostToDevice);
        free(ds);
    }
    DevState s0;
    memset(&s0, 0, sizeof s0);
    s0.gain = 1.0;
    s0.amb_r = -1;
    if (e == cudaSuccess) e = cudaMemcpy(h->st, &s0, sizeof s0, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        rx_destroy(h);
        return RX_ECUDA;
    }
    h->ebase_cur = -kEHist;
    h->ybase_cur = -kYHist;
    *out = h;
    return RX_OK;
}

rx_status rx_process(rx_handle *h, const uint8_t *in, uint8_t *bits_out, void *stream, int64_t *nbits_out)
{
    if (!h || !in || !nbits_out) return RX_EINVAL;
    if (h->broken) return RX_ESTATE;
    if (((uintptr_t)in) & 15) return RX_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const rx_config &c = h->cfg;
    Sched s = schedule(h, h->calls, h->q_prev);
    long long base = h->calls * h->nb;
    long long sym_lo = h->trained ? h->q_prev : 0;
    bool do_train = !h->trained && s.q_k >= c.ntrain && s.q_k > 0;
    long long pay_lo = do_train ? c.ntrain : h->q_prev;
    long long npay = (h->trained || do_train) ? s.q_k - pay_lo : 0;
    if (npay > 0 && !bits_out) return RX_EINVAL;
    cudaError_t e = cudaSuccess;
    int par = (int)(h->calls & 1);

    if (h->prof_on && h->prof_head - h->prof_tail >= kProfRing) prof_harvest_one(h);
    prof_mark(h, 0, st);
    // 12-bit unpack into [history | buffer]: the PAM chain's input; the KK kernels
    // read the packed bytes themselves, so there it only feeds the debug view
    if (!h->kk || c.debug) {
        int cw_new = h->cw ^ 1;
        e = launch_unpack(in, h->codes[cw_new], h->codes[h->cw], h->nb, h->nhist, h->nb, h->calls == 0,
                          c.pack_order, h->kk ? nullptr : &h->st->pam_s1[par],
                          h->kk ? nullptr : &h->st->pam_s2[par], st);
        h->cw = cw_new;
    }
    KkInput kin;
    if (h->kk) {
        kin.hist = h->phist[h->hw];
        kin.in = in;
        kin.hist_next = h->phist[h->hw ^ 1];
        kin.hist_bytes = (long long)h->nhist * 3 / 2;
        kin.in_bytes = h->nb * 3 / 2;
        kin.order = c.pack_order;
        kin.first_call = h->calls == 0;
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
        int ew_new = h->ew ^ 1;
        KkTables tb = {h->lnt, h->sqt, h->twN, h->twN2};
        e = launch_kk_front(g, kin, h->fftws, tb, h->E[ew_new], h->E[h->ew], h->partials, h->st, st,
                            h->prof_on ? h : nullptr);
        h->ew = ew_new;
        h->ebase_cur = g.ebase;
    } else if (e == cudaSuccess && h->kk) {
        e = launch_kk_hist(kin, st);
    }
    if (h->kk) h->hw ^= 1;
    // matched filter
    prof_mark(h, 4, st);
    if (e == cudaSuccess && s.f_k > h->f_prev) {
        long long yb = 2 * h->q_prev - kYHist;
        int yw_new = h->yw ^ 1;
        if (h->kk)
            e = launch_kk_mf(h->E[h->ew], h->ebase_cur, s.e_k, h->f_prev, s.f_k, h->rrc, h->hmf, h->ds_tab, c.ds_num,
                             c.ds_den, h->st, (float2 *)h->Y[yw_new], yb, (const float2 *)h->Y[h->yw], h->ybase_cur,
                             st, h->rrc_host);
        else
            e = launch_pam_mf(h->codes[h->cw], cbase, h->nb, s.avail, h->f_prev, s.f_k, h->rrc, h->hmf, h->st, par,
                              (float *)h->Y[yw_new], yb, (const float *)h->Y[h->yw], h->ybase_cur, st);
        h->yw = yw_new;
        h->ybase_cur = yb;
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
    prof_mark(h, 5, st);
    if (e == cudaSuccess && do_train) {
        e = launch_eq(h->ep, g, 1, h->Y[h->yw], h->taps[h->tw], nullptr, h->dec, h->winb, h->winrec, nullptr,
                      h->dbg_z, h->prbs, h->prbs_bits, h->st, st);
        h->trained = 1;
    }
    if (e == cudaSuccess && g.nblk > 0) {
        if (h->cnn) {
            // learned equaliser: one segment per payload window
            long long seg_base = 2 * pay_lo - 12 - h->ybase_cur;
            e = launch_cnn_decide(rx_cnn_dev_params(h->cnn), rx_cnn_dev_params_bf16(h->cnn),
                                  (const float2 *)h->Y[h->yw], seg_base, g.nwin, h->dec, h->winb, h->winrec,
                                  h->prbs_bits, pay_lo, h->ep.scale, h->mq, st);
        } else {
            e = launch_eq(h->ep, g, 0, h->Y[h->yw], h->taps[h->tw], h->taps[h->tw ^ 1], h->dec, h->winb, h->winrec,
                          h->dbg_win, h->dbg_z, h->prbs, h->prbs_bits, h->st, st);
            h->tw ^= 1;
        }
        prof_mark(h, 6, st);
        if (e == cudaSuccess) {
            int resolve = h->kk && !h->amb_done;
            e = launch_demap(h->ep, g, resolve, h->uw, h->dec, h->winb, h->winrec, h->dbg_win, bits_out, h->st, st);
            if (h->kk) h->uw ^= 1;
            h->amb_done = 1;
        }
    }
    if (h->prof_on) {
        prof_mark(h, kStages, st);
        h->prof_head++;
    }
    if (e != cudaSuccess) {
        h->broken = 1;
        return RX_ECUDA;
    }
    h->l_e_prev = h->e_prev;
    h->l_e_k = s.e_k;
    h->l_f_prev = h->f_prev;
    h->l_f_k = s.f_k;
    h->l_sym_lo = sym_lo;
    h->l_pay_lo = pay_lo;
    h->l_q_k = s.q_k;
    h->l_nwin = g.nwin;
    h->e_prev = s.e_k;
    h->f_prev = s.f_k;
    h->q_prev = s.q_k;
    h->calls++;
    *nbits_out = npay > 0 ? (long long)h->bps * npay : 0;
    return RX_OK;
}

rx_status rx_process_host(rx_handle *h, const uint8_t *host_in, uint8_t *host_bits_out, void *stream,
                          int64_t *nbits_out)
{
    if (!h || !host_in || !host_bits_out || !nbits_out) return RX_EINVAL;
    if (h->broken) return RX_ESTATE;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(h->in_stage, host_in, (size_t)(h->nb * 3 / 2), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return RX_ECUDA;
    rx_status r = rx_process(h, h->in_stage, h->bits_stage, stream, nbits_out);
    if (r != RX_OK) return r;
    if (*nbits_out > 0 &&
        cudaMemcpyAsync(host_bits_out, h->bits_stage, (size_t)((*nbits_out + 7) / 8), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
        return RX_ECUDA;
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
    o->calls = h->calls;
    o->samples = h->calls * h->nb;
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
        src = h->dec;
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
        double v[5] = {s.carrier_re, s.carrier_im, s.gain, s.pam_mu, s.pam_inv_sd};
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
    if (!h) return RX_EINVAL;
    if (enable && !h->prof_ev) {
        h->prof_ev = (cudaEvent_t *)calloc((size_t)kProfRing * kStages1, sizeof(cudaEvent_t));
        h->prof_used = (int *)calloc(kProfRing, sizeof(int));
        if (!h->prof_ev || !h->prof_used) return RX_ENOMEM;
        for (int i = 0; i < kProfRing * kStages1; i++)
            if (cudaEventCreate(&h->prof_ev[i]) != cudaSuccess) return RX_ECUDA;
    }
    h->prof_on = enable ? 1 : 0;
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

rx_status rx_set_cnn(rx_handle *h, const rx_cnn *cnn)
{
    if (!h || (cnn && !h->kk)) return RX_EINVAL;
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
