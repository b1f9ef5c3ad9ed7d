// Internal declarations shared by the receiver's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rx.h"

namespace rxk {

// ------------------------------------------------------------------ constants
constexpr int kWin = 64;          // symbols per window (one warp: two per lane)
constexpr int kMaxTaps = 31;      // adaptive FIR taps, one per lane
constexpr int kYHist = 16;        // 2-sps samples of equaliser history before a block
constexpr int kEHist = 1024;      // ADC samples of field history kept for the MF (>= fd_n)
constexpr int kPamHist = 64;      // codes kept before a PAM buffer (>= 2 * MF half length)
constexpr int kCtaK1 = 256;       // threads per K1a / K1c CTA
constexpr int kEqWarpsMax = 8;    // most warps (equaliser blocks) per K3 CTA
constexpr int kWaitLimit = 1 << 22;   // bounded mbarrier polls before flagging RX_ETIMEOUT
constexpr int kSlots = 3;
constexpr int kInSlots = 4;     // device staging slots of host input buffers (copies run up to 3 calls ahead)
constexpr int kMaxEqBlock = 4096;  // largest eq_block (symbols)
constexpr int kPrbsWords = 1040;   // PRBS-15 period + 256 bits, bit-packed MSB first

// counters in DevState::cnt
enum { C_SYMBOLS, C_BITS, C_BITERR, C_RAWERR, C_SYMERR, C_SLIP, C_NEAR, C_AMBIG, C_WINDOWS, C_NCNT };

// clock tracker across calls: unwrap carry (last unwrapped delay and its offset)
// and least-squares sums of the unwrapped block delays since the last reset
struct ClockTrack {
    int have, pad;
    long long n;
    double y, off, x0, sx, sy, sxx, sxy;
};

// device-resident state of one stream
struct DevState {
    ClockTrack ck;
    unsigned long long cnt[C_NCNT];
    double cg[kSlots][4];                  // KK per slot: carrier re, carrier im, gain
    double cg_flush[4];                    // KK: carrier and gain of the last real buffer (flush)
    double pam_mu, pam_inv_sd;             // PAM: this call's normalisation (debug view)
    long long pam_s1[3], pam_s2[3];        // PAM: integer sums of codes / codes^2, by call index mod 3
    int unwrap_have[2], unwrap_b[2];       // pi/2 unwrap carry, by parity
    int diff_have[2], diff_q[2];           // differential coding: quadrant of the last symbol, by parity
    long long unwrap_m[2];
    int amb_r;                             // stream-start rotation, -1 before
    int first_code;                        // 12-bit code of the stream's first sample
    unsigned long long csum[kSlots][3];    // KK per slot: carrier sums (re, im in 2^-24) and sum of 2I
    unsigned int ticket[kSlots];           // last-CTA ticket of the carrier reduction, per slot
    unsigned int eq_ticket;                // last-warp ticket of the frozen form's tap step
    int err;                               // RX_ETIMEOUT when a bounded wait ran out
};

// Per-buffer latency record on the device clock (%globaltimer, ns).  A recorded
// call owns slot (its index mod kLatSlots): its first kernel stamps t0 and clears t1,
// every CTA of its demap raises t1 to its own end time (one relaxed atomic, no
// fence), and the record is binned when the slot is next taken (by the first kernel
// of the call kLatSlots recorded calls later, which stream order puts after that
// demap) or by rx_stats, which bins and clears every slot still holding one.
// kLatSlots is far more than the calls the pipeline holds in flight (its slot rings
// bound that to about three times kSlots).
constexpr int kLatSlots = 64;
constexpr int kLatBins = 65536;
constexpr unsigned long long kLatBinNs = 500;
struct LatSlot {
    unsigned long long t0, t1;
};
struct LatRecord {
    LatSlot slot[kLatSlots];
    unsigned long long n, miss, max_ns, budget_ns;
    unsigned int hist[kLatBins];
};
__device__ __forceinline__ unsigned long long dev_clock_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bin a finished record (t1 > t0 > 0) into the histogram and counters
__device__ __forceinline__ void lat_bin(LatRecord *r, unsigned long long t0, unsigned long long t1)
{
    if (!(t0 && t1 > t0)) return;
    const unsigned long long d = t1 - t0;
    unsigned long long b = d / kLatBinNs;
    if (b >= (unsigned long long)kLatBins) b = kLatBins - 1;
    atomicAdd(&r->hist[b], 1u);
    atomicAdd(&r->n, 1ull);
    if (d > r->budget_ns) atomicAdd(&r->miss, 1ull);
    atomicMax(&r->max_ns, d);
}
// one thread of the call's first kernel, at its start: stamp the slot, then bin the
// record the slot held
__device__ __forceinline__ void lat_start(LatRecord *r, int slot)
{
    LatSlot *s = &r->slot[slot];
    const unsigned long long o0 = s->t0, o1 = s->t1;
    s->t0 = dev_clock_ns();
    s->t1 = 0ull;
    lat_bin(r, o0, o1);
}
// thread 0 of every CTA of the call's last kernel, after its CTA's work
__device__ __forceinline__ void lat_end(LatRecord *r, int slot)
{
    atomicMax(&r->slot[slot].t1, dev_clock_ns());
}
// rx_stats: bin and clear every slot (one thread per slot)
cudaError_t launch_lat_flush(LatRecord *r, cudaStream_t st);

// per-call geometry of the KK overlap-save blocks
struct KkGeom {
    long long e_prev, e_k;     // KK outputs emitted: [e_prev, e_k)
    long long avail;           // stream samples seen after this buffer
    long long cbase;           // stream index of codes[0]
    long long ebase;           // stream index of field workspace [0] (= e_prev - kEHist)
    long long ebase_prev;      // same for the previous field workspace
    int N, V, hop, J, npairs, N2;
    int sps;
    int slot;                  // carrier / gain slot written by this call
    int fused;                 // 2^16-point blocks: one cluster kernel instead of three
};

// constant tables of the KK front end (device pointers).  Twiddles of an M-point
// transform are factored W_M^a = hi[a >> s] * lo[a & (2^s - 1)], s = ceil(log2(M)/2),
// stored as [lo (2^s) | hi (M / 2^s)].
struct KkTables {
    const float *lnt;      // 4096: ln(I)/2 - ln(2048)/2, I = code (0.5 for code 0)
    const float2 *twN;     // factored W_N
    const float2 *twN2;    // factored W_{N/16}
};
constexpr int kLutCodes = 4096;
// number of float2 entries of the factored table of an M-point transform
int kk_tw_entries(int M);
// host: fill the tables of a KK front end with FFT length N
void kk_host_tables(int N, float *lnt, float2 *twN, float2 *twN2);

// packed input of one KK call
struct KkInput {
    const uint8_t *hist;     // packed samples [base - nhist, base)
    const uint8_t *in;       // packed buffer
    uint8_t *hist_next;      // receives packed samples [avail - nhist, avail), or null
    long long hist_bytes, in_bytes;
    int order, first_call;
    LatRecord *lat;          // latency record whose slot this call's first kernel stamps, or null
    int lat_slot;
};

// per-call schedule of the equaliser
struct EqGeom {
    long long sym_lo;          // first symbol processed (0 on the training call)
    long long pay_lo;          // first payload symbol
    long long q_k;             // symbols processed up to (exclusive)
    long long ybase;           // stream index (2-sps) of Y workspace [0]
    int nblk;                  // payload blocks in this call
    int nwin;                  // payload windows in this call
    float2 *gpart;             // frozen form: per-window tap-gradient partials of the last block
    long long score_end;       // windows reaching symbol score_end or beyond are not scored
    LatRecord *lat;            // latency record the demap closes for this call, or null
    int lat_slot;
};

struct EqParams {
    int kk, mq, bps, ntaps, th, win, eq_block, ntrain, ncma, bps_b, amb_syms;
    float scale, r2, mu, mu_train, mu_cma;
    int frozen;   // payload blocks filter with the call's start taps (block-Toeplitz form)
    int diff;     // differentially quadrant-coded QAM: decode and score quadrant differences
    int warps;    // equaliser blocks (warps) per CTA
    int dd;       // KK: the short decision-directed LMS updated symbol by symbol, no phase search
};

// ------------------------------------------------------------------ launchers
// (each returns cudaGetLastError() after enqueuing)
cudaError_t launch_unpack(const uint8_t *in, uint16_t *codes, const uint16_t *codes_prev,
                          long long nb, int nhist, long long prev_off, int first_call,
                          int pack_order, long long *s1, long long *s2, cudaStream_t st,
                          LatRecord *lat = nullptr, int lat_slot = 0);

// copy of the next call's packed history only (calls that emit no field)
// Cross-stream order of the front end when consecutive calls run on different
// streams (null events: one stream, nothing to do): the forward pass waits for
// wait_fwd (the previous call's history copy) and records rec_fwd after its own;
// the inverse pass waits for wait_inv (the previous call's field, whose tail it
// carries as history).
struct KkSync {
    cudaEvent_t wait_fwd, rec_fwd, wait_inv;
};
cudaError_t launch_kk_hist(const KkInput &inp, cudaStream_t st, const KkSync &sync);

cudaError_t launch_kk_front(const KkGeom &g, const KkInput &inp, float2 *fftws, const KkTables &tb,
                            float2 *E, const float2 *E_prev, DevState *dst, cudaStream_t st, void *prof,
                            const KkSync &sync);
// stage-boundary hook of the profiler (defined with the C ABI; prof may be null)
void prof_stage(void *prof, int stage, cudaStream_t st);

cudaError_t launch_kk_mf(const float2 *E, long long ebase, long long e_k, long long f_prev,
                         long long f_k, const float *rrc, int hmf, const float2 *ds_tab,
                         int ds_num, int ds_den, const double *cg, float2 *Y, long long ybase,
                         const float2 *Y_prev, long long ybase_prev, cudaStream_t st,
                         const float *rrc_host);

// resampler of the KK field to the transmitter's grid: outputs [r_prev, r_k) at ADC
// positions (i0 2^32 + f0 + (m - r_prev) step) / 2^32; tab: 1024 x 16 taps
cudaError_t launch_kk_resample(const float2 *E, long long ebase, long long r_prev, long long r_k, long long i0,
                               unsigned f0, long long step, const float *tab, float2 *R, long long rbase,
                               const float2 *R_prev, long long rbase_prev, cudaStream_t st);

// frequency-domain form (static filter on N-point overlap-save blocks, hop N/2,
// N/2-point bin-truncation inverse); f_prev and f_k are multiples of N/4; clk (or
// null) receives each block's band-edge clock correlation over |k - N/8| <= w
cudaError_t launch_kk_fdmf(const float2 *E, long long ebase, long long f_prev, long long f_k, int N,
                           const float2 *H, const float2 *tw, const float2 *ds_tab, int ds_num, int ds_den,
                           const double *cg, float2 *Y, long long ybase, const float2 *Y_prev,
                           long long ybase_prev, cudaStream_t st, float2 *clk, int w);

// PAM frequency-domain form, 1024-point blocks (hop 512) at the input rate;
// f_prev and f_k are multiples of 512
cudaError_t launch_pam_fd1024(const uint16_t *codes, long long cbase, long long nb, long long n_end,
                              long long f_prev, long long f_k, const float2 *H, const float2 *tw, DevState *dst,
                              int parity, float *Y, long long ybase, const float *Y_prev, long long ybase_prev,
                              cudaStream_t st, float2 *clk, int wbin);

// PAM with the resampler: the call's normalised codes for [cbase, n_end) as a complex
// series (imaginary 0), then the matched filter on the resampled series
cudaError_t launch_pam_norm(const uint16_t *codes, long long cbase, long long nb, long long n_end, DevState *dst,
                            int parity, float2 *X, cudaStream_t st);
cudaError_t launch_pam_mf_r(const float2 *R, long long rbase, long long f_prev, long long f_k, const float *rrc, int hmf,
                            float *Y, long long ybase, const float *Y_prev, long long ybase_prev, cudaStream_t st);

cudaError_t launch_pam_mf(const uint16_t *codes, long long cbase, long long nb, long long n_end, long long f_prev,
                          long long f_k, const float *rrc, int hmf, DevState *dst, int parity,
                          float *Y, long long ybase, const float *Y_prev, long long ybase_prev,
                          cudaStream_t st);

// zin: soft symbols of the payload from the block-Toeplitz tensor-core FIR
// (frozen form), or null to filter in FP32 inside the equaliser
cudaError_t launch_eq(const EqParams &p, const EqGeom &g, int train, const void *Y, const float2 *zin,
                      float2 *taps_in, float2 *taps_out, uint8_t *dec, uint8_t *winb, uint4 *winrec,
                      float4 *dbg_win, float2 *dbg_z, const uint8_t *prbs, const uint32_t *prbs_bits,
                      DevState *dst, cudaStream_t st);

// block-Toeplitz FIR on the tensor cores (frozen taps): z[k - k_lo] for
// k in [k_lo, k_lo + nsym), z_k = sum_i conj(w_i) Y[2k + TH - i - ybase]
cudaError_t launch_fir_tc(int prec, const float2 *Y, long long ybase, long long k_lo, long long nsym,
                          const float2 *taps, int ntaps, int scale_block, float2 *z, int *err, int nsm,
                          cudaStream_t st);

// one-time kernel attributes (dynamic shared memory above 48 KB) of what a handle
// launches, set at creation so that launches and graph captures make no such calls
cudaError_t prepare_eq(const EqParams &p);
size_t eq_smem_bytes(const EqParams &p, int warps);   // dynamic shared memory of a payload CTA
constexpr size_t kMaxSmemCta = 227 * 1024;
cudaError_t prepare_fir_tc(int prec);
cudaError_t prepare_kk_front();

cudaError_t launch_demap(const EqParams &p, const EqGeom &g, int resolve_amb, int uw_in,
                         const uint8_t *dec, const uint8_t *winb, const uint4 *winrec, float4 *dbg_win,
                         uint8_t *bits_out, const uint32_t *prbs_bits, DevState *dst, cudaStream_t st);

// CNN decisions for nseg consecutive payload windows (receiver mode)
// CNN receiver on the tensor cores: soft symbols and decisions of nwin 64-symbol
// windows; y[seg_base + 2 j - 12 ..] feeds symbol j, inputs at y_end and beyond read 0
cudaError_t launch_cnn_decide(const float *prm, const float2 *y, long long seg_base, long long y_end,
                              int nwin, uint8_t *dec, uint8_t *winb, uint4 *winrec, const uint32_t *prbs_bits,
                              long long k_first, float scale, int mq, float2 *soft, int *err, int nsm, cudaStream_t st,
                              int bf16);
cudaError_t prepare_cnn_rx();

}  // namespace rxk

extern "C" {
const float *rx_cnn_dev_params(const rx_cnn *c);
}
