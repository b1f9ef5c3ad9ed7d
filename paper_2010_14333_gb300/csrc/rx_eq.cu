// Adaptive FIR equaliser with blind phase search (K3) and the decision / pi/2
// unwrap / Gray demap / bit-error kernel (K4).
//
// Paper: Sec. 2 -- after reduction to 2 samples/symbol a decision-directed LMS
// equaliser performs symbol-phase recovery, decision and demapping, and these
// operations run for the data blocks of each buffer in parallel; the PAM chain
// ends with symbol decision and demapping (Fig. 1b, 1c).  Q-factor from BER, Sec. 3.
//
// Block-parallel semantics: every equaliser block of eq_block symbols starts from
// the same taps (those left by the last block of the previous call, or by the
// sequential training at stream start) and adapts on its own, window by window:
// filter the window's 64 symbols, pick the phase by blind phase search (QAM),
// decide, form the errors and apply one block-LMS update after the window.
// One warp runs one block: lane b tests phase b in the search (argmin by warp
// shuffle), lanes hold two symbols each in the filter and one tap each in the
// update.  A block's 2-sps input is staged into shared memory by one bulk
// asynchronous copy (cp.async.bulk, completion on an mbarrier).
#include <type_traits>

#include "rx_common.cuh"
#include "rx_internal.cuh"

namespace rxk {

// ------------------------------------------------------------ bulk copy / mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// bounded wait on phase `parity`; false when the poll limit ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    for (int it = 0; it < kWaitLimit; it++) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(smem_u32(bar)), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// ------------------------------------------------------------- symbol helpers
__device__ __forceinline__ int decide(float t, int mq)
{
    int L = 0;
    for (int j = 0; j < mq - 1; j++) L += (t >= (float)(2 * j - (mq - 2)));
    return L;
}
__device__ __forceinline__ bool near_thr(float t, int mq)
{
    bool n = false;
    for (int j = 0; j < mq - 1; j++) n |= fabsf(t - (float)(2 * j - (mq - 2))) < 1e-4f;
    return n;
}
__device__ __forceinline__ float level(int L, int mq) { return (float)(2 * L - (mq - 1)); }
// squared distance to the nearest odd-integer level by folding: for 4 levels
// (||t| - 2| - 1)^2, for 2 levels (|t| - 1)^2
__device__ __forceinline__ float dist_fold(float t, int mq)
{
    float a = fabsf(t);
    for (int h = mq >> 1; h > 1; h >>= 1) a = fabsf(a - (float)h);
    a -= 1.f;
    return a * a;
}
__device__ __forceinline__ int gray(int L) { return L ^ (L >> 1); }
__device__ __forceinline__ int gray_inv(int g)
{
    int L = g;
    for (int s = g >> 1; s; s >>= 1) L ^= s;
    return L;
}
// transmitted level indices of symbol k from the PRBS-15 table (MSB first)
__device__ __forceinline__ void tx_sym(const uint8_t *prbs, long long k, int bps, bool qam, int &LI, int &LQ)
{
    int nb = qam ? bps / 2 : bps;
    long long b0 = (long long)bps * k;
    int gi = 0, gq = 0;
    for (int t = 0; t < nb; t++) gi = (gi << 1) | prbs[(b0 + t) % 32767];
    if (qam)
        for (int t = 0; t < nb; t++) gq = (gq << 1) | prbs[(b0 + nb + t) % 32767];
    LI = gray_inv(gi);
    LQ = qam ? gray_inv(gq) : 0;
}
// rotate a level-index pair by -j (multiply the symbol by -j) q times
__device__ __forceinline__ void rot_levels(int &LI, int &LQ, int q, int mq)
{
    for (int s = 0; s < (q & 3); s++) {
        int t = LI;
        LI = LQ;
        LQ = mq - 1 - t;
    }
}

// ---------------------------------------------------------------- one window
// ys: 2-sps input with ys[i] = y[ym0 + i]; the window's first symbol is k0.
// mode: 0 CMA, 1 data-aided (PAM training), 2 decision directed.
// Returns the window's b* (QAM DD) or -1.
struct WinOut {
    int b;
    float best, second;
};

__device__ __forceinline__ WinOut qam_window(const EqParams &p, const float2 *ys, long long ym0,
                                             long long k0, float2 *zs, float2 *es, float2 *ws, int mode,
                                             float mu, int lane, uint8_t *dec_out, float2 *dbg_z)
{
    const int th = p.th;
    // filter: z_k = sum_i conj(w_i) y[2k - i]
#pragma unroll
    for (int h = 0; h < 2; h++) {
        int q = lane + 32 * h;
        const float2 *yc = ys + (2 * (k0 + q) - ym0);
        float ar = 0.f, ai = 0.f;
        for (int i = 0; i < p.ntaps; i++) {
            float2 w = ws[i], y = yc[th - i];
            ar = fmaf(w.x, y.x, fmaf(w.y, y.y, ar));
            ai = fmaf(w.x, y.y, fmaf(-w.y, y.x, ai));
        }
        zs[q] = make_float2(ar, ai);
        if (dbg_z) dbg_z[q] = make_float2(ar, ai);
    }
    __syncwarp();
    WinOut R;
    R.b = -1;
    R.best = 0.f;
    R.second = 0.f;
    float cs = 1.f, sn = 0.f;   // cos / sin of the chosen phase
    if (mode == 2) {
        // blind phase search, lane b tests theta_b = (b/B)(pi/2) - pi/4
        float tsn, tcs;
        sincospif((float)lane / (float)(2 * p.bps_b) - 0.25f, &tsn, &tcs);
        float sc = p.scale * tcs, ss = p.scale * tsn;
        float M = 0.f;
        for (int q = 0; q < kWin; q++) {
            float2 z = zs[q];
            float vr = fmaf(z.x, sc, z.y * ss);
            float vi = fmaf(z.y, sc, -z.x * ss);
            M += dist_fold(vr, p.mq) + dist_fold(vi, p.mq);
        }
        if (lane >= p.bps_b) M = __int_as_float(0x7f800000);
        float m1 = M, m2 = __int_as_float(0x7f800000);
        int b1 = lane;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            float om1 = __shfl_xor_sync(0xffffffffu, m1, o);
            float om2 = __shfl_xor_sync(0xffffffffu, m2, o);
            int ob1 = __shfl_xor_sync(0xffffffffu, b1, o);
            if (om1 < m1 || (om1 == m1 && ob1 < b1)) {
                m2 = fminf(m1, om2);
                m1 = om1;
                b1 = ob1;
            } else {
                m2 = fminf(m2, om1);
            }
        }
        R.b = b1;
        R.best = m1;
        R.second = m2;
        cs = __shfl_sync(0xffffffffu, tcs, b1);
        sn = __shfl_sync(0xffffffffu, tsn, b1);
    }
    // decisions and errors
    const float inv_s = 1.0f / p.scale;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        int q = lane + 32 * h;
        float2 z = zs[q];
        float vr = p.scale * fmaf(z.x, cs, z.y * sn);
        float vi = p.scale * fmaf(z.y, cs, -z.x * sn);
        int LI = decide(vr, p.mq), LQ = decide(vi, p.mq);
        bool nr = near_thr(vr, p.mq) || near_thr(vi, p.mq);
        if (dec_out) dec_out[q] = (uint8_t)(LI | (LQ << 3) | (nr ? 64 : 0));
        float2 e;
        if (mode == 0) {
            float f = p.r2 - (z.x * z.x + z.y * z.y);
            e = make_float2(z.x * f, z.y * f);
        } else {
            float dI = level(LI, p.mq) * inv_s, dQ = level(LQ, p.mq) * inv_s;
            e = make_float2(fmaf(dI, cs, -dQ * sn) - z.x, fmaf(dI, sn, dQ * cs) - z.y);
        }
        es[q] = e;
    }
    __syncwarp();
    // block-LMS update after the window: w_i += mu sum_k y[2k - i] conj(e_k)
    if (lane < p.ntaps) {
        int off = lane - th;
        float gr = 0.f, gi = 0.f;
        const float2 *yb = ys + (2 * k0 - ym0 - off);
        for (int q = 0; q < kWin; q++) {
            float2 y = yb[2 * q], e = es[q];
            gr = fmaf(y.x, e.x, fmaf(y.y, e.y, gr));
            gi = fmaf(y.y, e.x, fmaf(-y.x, e.y, gi));
        }
        float2 w = ws[lane];
        ws[lane] = make_float2(fmaf(mu, gr, w.x), fmaf(mu, gi, w.y));
    }
    __syncwarp();
    return R;
}

__device__ __forceinline__ void pam_window(const EqParams &p, const float *ys, long long ym0, long long k0,
                                           float *zs, float *es, float *ws, int mode, float mu, int lane,
                                           uint8_t *dec_out, float2 *dbg_z, const uint8_t *prbs)
{
    const int th = p.th;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        int q = lane + 32 * h;
        const float *yc = ys + (2 * (k0 + q) - ym0);
        float a = 0.f;
        for (int i = 0; i < p.ntaps; i++) a = fmaf(ws[i], yc[th - i], a);
        zs[q] = a;
        if (dbg_z) dbg_z[q] = make_float2(a, 0.f);
        int L = decide(a, p.mq);
        bool nr = near_thr(a, p.mq);
        if (dec_out) dec_out[q] = (uint8_t)(L | (nr ? 64 : 0));
        float d;
        if (mode == 1) {
            int aI, aQ;
            tx_sym(prbs, k0 + q, p.bps, false, aI, aQ);
            d = level(aI, p.mq);
        } else {
            d = level(L, p.mq);
        }
        es[q] = d - a;
    }
    __syncwarp();
    if (lane < p.ntaps) {
        int off = lane - th;
        const float *yb = ys + (2 * k0 - ym0 - off);
        float g = 0.f;
        for (int q = 0; q < kWin; q++) g = fmaf(yb[2 * q], es[q], g);
        ws[lane] = fmaf(mu, g, ws[lane]);
    }
    __syncwarp();
}

// -------------------------------------------------------------- equaliser kernel
// Payload: one warp per block of eq_block symbols, input staged by one bulk copy.
// Training (train=1): one warp runs the training windows sequentially, staging
// each window's input with plain loads.
template <bool QAM>
__global__ void k_eq(EqParams p, EqGeom g, int train, const void *__restrict__ Yv, float2 *taps_in,
                     float2 *taps_out, uint8_t *__restrict__ dec, uint8_t *__restrict__ winb,
                     float4 *__restrict__ dbg_win, float2 *__restrict__ dbg_z, const uint8_t *__restrict__ prbs,
                     DevState *dst)
{
    typedef typename std::conditional<QAM, float2, float>::type T;
    extern __shared__ __align__(16) unsigned char smraw[];
    const T *Y = reinterpret_cast<const T *>(Yv);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int B = train ? kWin : p.eq_block;
    const int ylen = 2 * B + 2 * kYHist;
    // per-warp shared layout: [mbarrier | y (ylen) | z (64) | e (64) | taps (32)]
    size_t per_warp = 16 + (size_t)(ylen + 2 * kWin + 32) * sizeof(T);
    per_warp = (per_warp + 15) & ~(size_t)15;
    unsigned char *base = smraw + per_warp * wid;
    uint64_t *bar = reinterpret_cast<uint64_t *>(base);
    T *ys = reinterpret_cast<T *>(base + 16);
    T *zs = ys + ylen;
    T *es = zs + kWin;
    T *ws = es + kWin;
    long long blk = (long long)blockIdx.x * kEqWarps + wid;
    if (!train && blk >= g.nblk) return;
    // start taps
    if (lane < p.ntaps) {
        if (QAM) reinterpret_cast<float2 *>(ws)[lane] = taps_in[lane];
        else reinterpret_cast<float *>(ws)[lane] = taps_in[lane].x;
    }
    unsigned ambig = 0;
    if (train) {
        for (long long k0 = 0; k0 < p.ntrain; k0 += kWin) {
            long long ym0 = 2 * k0 - kYHist;
            for (int i = lane; i < ylen; i += 32) ys[i] = Y[ym0 + i - g.ybase];
            __syncwarp();
            float2 *dz = dbg_z ? dbg_z + (k0 - g.sym_lo) : nullptr;
            if (QAM) {
                int mode = (k0 < p.ncma) ? 0 : 2;
                float mu = mode == 0 ? p.mu_cma : p.mu;
                qam_window(p, reinterpret_cast<float2 *>(ys), ym0, k0, reinterpret_cast<float2 *>(zs),
                           reinterpret_cast<float2 *>(es), reinterpret_cast<float2 *>(ws), mode, mu, lane,
                           nullptr, dz);
            } else {
                pam_window(p, reinterpret_cast<float *>(ys), ym0, k0, reinterpret_cast<float *>(zs),
                           reinterpret_cast<float *>(es), reinterpret_cast<float *>(ws), 1, p.mu_train, lane,
                           nullptr, dz, prbs);
            }
        }
        if (lane < p.ntaps)
            taps_in[lane] = QAM ? reinterpret_cast<float2 *>(ws)[lane]
                                : make_float2(reinterpret_cast<float *>(ws)[lane], 0.f);
        return;
    }
    long long kb = g.pay_lo + blk * B;
    long long ym0 = 2 * kb - kYHist;
    if (lane == 0) {
        mbar_init(bar, 1);
        unsigned bytes = (unsigned)(ylen * sizeof(T));
        mbar_expect_tx(bar, bytes);
        bulk_g2s(ys, Y + (ym0 - g.ybase), bytes, bar);
    }
    __syncwarp();
    if (!mbar_wait(bar, 0)) {
        if (lane == 0) atomicExch(&dst->err, (int)RX_ETIMEOUT);
        mbar_wait(bar, 0);
        return;
    }
    for (int w = 0; w < B / kWin; w++) {
        long long k0 = kb + (long long)w * kWin;
        uint8_t *dq = dec + (k0 - g.pay_lo);
        float2 *dz = dbg_z ? dbg_z + (k0 - g.sym_lo) : nullptr;
        long long wi = (k0 - g.pay_lo) / kWin;
        if (QAM) {
            WinOut R = qam_window(p, reinterpret_cast<float2 *>(ys), ym0, k0, reinterpret_cast<float2 *>(zs),
                                  reinterpret_cast<float2 *>(es), reinterpret_cast<float2 *>(ws), 2, p.mu, lane,
                                  dq, dz);
            if (lane == 0) {
                winb[wi] = (uint8_t)R.b;
                if (dbg_win) dbg_win[wi] = make_float4((float)R.b, 0.f, R.best, R.second);
                ambig += (R.second - R.best) <= 1e-6f * R.best;
            }
        } else {
            pam_window(p, reinterpret_cast<float *>(ys), ym0, k0, reinterpret_cast<float *>(zs),
                       reinterpret_cast<float *>(es), reinterpret_cast<float *>(ws), 2, p.mu, lane, dq, dz, prbs);
            if (lane == 0) winb[wi] = 0;
        }
    }
    if (blk == g.nblk - 1 && lane < p.ntaps)
        taps_out[lane] = QAM ? reinterpret_cast<float2 *>(ws)[lane]
                             : make_float2(reinterpret_cast<float *>(ws)[lane], 0.f);
    if (lane == 0 && ambig) atomicAdd(&dst->cnt[C_AMBIG], (unsigned long long)ambig);
}

static size_t eq_smem_per_warp(bool qam, int B)
{
    size_t el = qam ? sizeof(float2) : sizeof(float);
    size_t w = 16 + (size_t)(2 * B + 2 * kYHist + 2 * kWin + 32) * el;
    return (w + 15) & ~(size_t)15;
}

cudaError_t launch_eq(const EqParams &p, const EqGeom &g, int train, const void *Y, float2 *taps_in,
                      float2 *taps_out, uint8_t *dec, uint8_t *winb, float4 *dbg_win, float2 *dbg_z,
                      const uint8_t *prbs, DevState *dst, cudaStream_t st)
{
    bool qam = p.kk != 0;
    if (train) {
        size_t smem = eq_smem_per_warp(qam, kWin);
        if (qam) k_eq<true><<<1, 32, smem, st>>>(p, g, 1, Y, taps_in, taps_out, dec, winb, dbg_win, dbg_z, prbs, dst);
        else k_eq<false><<<1, 32, smem, st>>>(p, g, 1, Y, taps_in, taps_out, dec, winb, dbg_win, dbg_z, prbs, dst);
        return cudaGetLastError();
    }
    size_t smem = eq_smem_per_warp(qam, p.eq_block) * kEqWarps;
    unsigned grid = (unsigned)((g.nblk + kEqWarps - 1) / kEqWarps);
    if (qam) {
        cudaFuncSetAttribute(k_eq<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_eq<true><<<grid, 32 * kEqWarps, smem, st>>>(p, g, 0, Y, taps_in, taps_out, dec, winb, dbg_win, dbg_z,
                                                      prbs, dst);
    } else {
        cudaFuncSetAttribute(k_eq<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_eq<false><<<grid, 32 * kEqWarps, smem, st>>>(p, g, 0, Y, taps_in, taps_out, dec, winb, dbg_win, dbg_z,
                                                       prbs, dst);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ demap / BER
// R windows per CTA.  The pi/2 unwrap counter of window w is the carried value
// plus a prefix sum of integer increments; each CTA sums the increments of all
// earlier windows itself (a few KB of window indices), then scans its own.
constexpr int kDemapWin = 64;
constexpr int kDemapThreads = 256;

__device__ __forceinline__ int unwrap_inc(int b_prev, int b, int B)
{
    int d = b_prev - b;
    return (d > B / 2) - (d < -B / 2);
}

template <bool QAM>
__global__ void __launch_bounds__(kDemapThreads)
    k_demap(EqParams p, EqGeom g, int resolve_amb, int uw_in, const uint8_t *__restrict__ dec,
            const uint8_t *__restrict__ winb, float4 *__restrict__ dbg_win, const uint8_t *__restrict__ prbs,
            uint8_t *__restrict__ bits_out, DevState *dst)
{
    __shared__ long long s_m[kDemapWin];
    __shared__ int s_red[kDemapThreads / 32][4];
    __shared__ int s_r;
    __shared__ uint32_t s_bits[kDemapThreads / 32][8];
    __shared__ unsigned long long s_cnt[C_NCNT];
    int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int w0 = blockIdx.x * kDemapWin;
    int wend = min(w0 + kDemapWin, g.nwin);
    if (tid < C_NCNT) s_cnt[tid] = 0;
    int have = 0, blast = 0;
    long long mstart = 0;
    if (QAM) {
        have = dst->unwrap_have[uw_in];
        blast = dst->unwrap_b[uw_in];
        mstart = have ? dst->unwrap_m[uw_in] : 0;
        // prefix of increments over windows [0, w0)
        int part = 0;
        for (int w = tid; w < w0; w += kDemapThreads) {
            int bp = (w == 0) ? blast : winb[w - 1];
            if (w > 0 || have) part += unwrap_inc(bp, winb[w], p.bps_b);
        }
        part = warp_sum_i(part);
        if (lane == 0) s_red[wid][0] = part;
        __syncthreads();
        long long pre = 0;
        for (int i = 0; i < kDemapThreads / 32; i++) pre += s_red[i][0];
        // inclusive scan of this CTA's increments (64 windows, two warps)
        int inc = 0;
        if (tid < kDemapWin && w0 + tid < wend) {
            int w = w0 + tid;
            int bp = (w == 0) ? blast : winb[w - 1];
            if (w > 0 || have) inc = unwrap_inc(bp, winb[w], p.bps_b);
        }
        int sc = inc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, sc, o);
            if (lane >= o) sc += v;
        }
        __syncthreads();
        if (tid == 31) s_red[0][1] = sc;
        __syncthreads();
        if (tid < kDemapWin) {
            long long tot = sc + ((tid >= 32) ? s_red[0][1] : 0);
            s_m[tid] = mstart + pre + tot;
        }
        // stream-start pi/2 ambiguity: every CTA resolves it identically
        if (resolve_amb) {
            __syncthreads();
            int nw = p.amb_syms / kWin;    // windows 0..nw-1 of this call
            __shared__ long long s_ma[64];
            if (tid < 32) {
                int acc = 0;
                long long mw[2];
                for (int h = 0; h < 2; h++) {
                    int w = lane + 32 * h;
                    int v = 0;
                    if (w < nw && w > 0) v = unwrap_inc(winb[w - 1], winb[w], p.bps_b);
                    // inclusive scan per half
                    int s2 = v;
                    for (int o = 1; o < 32; o <<= 1) {
                        int t = __shfl_up_sync(0xffffffffu, s2, o);
                        if (lane >= o) s2 += t;
                    }
                    mw[h] = acc + s2;
                    acc += __shfl_sync(0xffffffffu, s2, 31);
                }
                s_ma[lane] = mw[0];
                s_ma[lane + 32] = mw[1];
            }
            __syncthreads();
            int cnt[4] = {0, 0, 0, 0};
            for (int s = tid; s < p.amb_syms; s += kDemapThreads) {
                uint8_t dv = dec[s];
                int aI, aQ;
                tx_sym(prbs, g.pay_lo + s, p.bps, true, aI, aQ);
                for (int r = 0; r < 4; r++) {
                    int LI = dv & 7, LQ = (dv >> 3) & 7;
                    rot_levels(LI, LQ, (int)((s_ma[s / kWin] + r) & 3), p.mq);
                    cnt[r] += (LI != aI) || (LQ != aQ);
                }
            }
            for (int r = 0; r < 4; r++) {
                int v = warp_sum_i(cnt[r]);
                if (lane == 0) s_red[wid][r] = v;
            }
            __syncthreads();
            if (tid == 0) {
                int best = 0;
                long long bc = -1;
                for (int r = 0; r < 4; r++) {
                    long long c = 0;
                    for (int i = 0; i < kDemapThreads / 32; i++) c += s_red[i][r];
                    if (bc < 0 || c < bc) { bc = c; best = r; }
                }
                s_r = best;
                if (blockIdx.x == 0) dst->amb_r = best;
            }
        } else if (tid == 0) {
            s_r = dst->amb_r;
        }
    }
    __syncthreads();
    const int r = QAM ? s_r : 0;
    const int nb = QAM ? p.bps / 2 : p.bps;
    const long long amb_end = QAM ? (long long)p.ntrain + p.amb_syms : 0;
    // one warp per window, two symbols per lane
    for (int wi = w0 + wid; wi < wend; wi += kDemapThreads / 32) {
        long long k0 = g.pay_lo + (long long)wi * kWin;
        long long mw = QAM ? s_m[wi - w0] : 0;
        if (dbg_win && lane == 0 && QAM) dbg_win[wi].y = (float)mw;
        if (lane < 8) s_bits[wid][lane] = 0u;
        __syncwarp();
        int ah[2][2], ref[2], nr = 0;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            int q = lane + 32 * h;
            uint8_t dv = dec[(k0 - g.pay_lo) + q];
            int LI = dv & 7, LQ = QAM ? ((dv >> 3) & 7) : 0;
            nr += (dv >> 6) & 1;
            if (QAM) rot_levels(LI, LQ, (int)((mw + r) & 3), p.mq);
            ah[h][0] = LI;
            ah[h][1] = LQ;
            int grp = QAM ? ((gray(LI) << nb) | gray(LQ)) : gray(LI);
            // output bits, MSB first, at bit offset q * bps of the window
            int bo = q * p.bps;
            for (int t = 0; t < p.bps; t++) {
                int bit = (grp >> (p.bps - 1 - t)) & 1;
                int pos = bo + t;
                if (bit) atomicOr(&s_bits[wid][pos >> 5], 1u << (31 - (pos & 31)));
            }
            long long kk = k0 + q, b0 = (long long)p.bps * kk;
            int rg = 0;
            for (int t = 0; t < p.bps; t++) rg = (rg << 1) | prbs[(b0 + t) % 32767];
            ref[h] = rg;
        }
        __syncwarp();
        int nbytes = 8 * p.bps;   // 64 symbols * bps bits / 8
        if (lane < nbytes) {
            uint32_t wv = s_bits[wid][lane >> 2];
            bits_out[(long long)wi * nbytes + lane] = (uint8_t)(wv >> (24 - 8 * (lane & 3)));
        }
        bool counted = !(QAM && k0 < amb_end);
        if (counted) {
            int nrot = QAM ? 4 : 1;
            int errs[4] = {0, 0, 0, 0}, serr[4] = {0, 0, 0, 0};
            for (int rho = 0; rho < nrot; rho++) {
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    int LI = ah[h][0], LQ = ah[h][1];
                    if (QAM) rot_levels(LI, LQ, rho, p.mq);
                    int grp = QAM ? ((gray(LI) << nb) | gray(LQ)) : gray(LI);
                    int ne = __popc(grp ^ ref[h]);
                    errs[rho] += ne;
                    serr[rho] += ne > 0;
                }
            }
            for (int rho = 0; rho < nrot; rho++) {
                errs[rho] = warp_sum_i(errs[rho]);
                serr[rho] = warp_sum_i(serr[rho]);
            }
            nr = warp_sum_i(nr);
            if (lane == 0) {
                int best = 0;
                for (int rho = 1; rho < nrot; rho++)
                    if (errs[rho] < errs[best]) best = rho;
                atomicAdd(&s_cnt[C_BITERR], (unsigned long long)errs[best]);
                atomicAdd(&s_cnt[C_RAWERR], (unsigned long long)errs[0]);
                atomicAdd(&s_cnt[C_SYMERR], (unsigned long long)serr[best]);
                atomicAdd(&s_cnt[C_SLIP], (unsigned long long)(best != 0));
                atomicAdd(&s_cnt[C_NEAR], (unsigned long long)nr);
                atomicAdd(&s_cnt[C_BITS], (unsigned long long)(p.bps * kWin));
                atomicAdd(&s_cnt[C_SYMBOLS], (unsigned long long)kWin);
            }
        }
        if (lane == 0) atomicAdd(&s_cnt[C_WINDOWS], 1ull);
    }
    __syncthreads();
    if (tid < C_NCNT && s_cnt[tid]) atomicAdd(&dst->cnt[tid], s_cnt[tid]);
    // carry the unwrap state to the next call
    if (QAM && wend == g.nwin && w0 < wend && tid == 0) {
        int o = uw_in ^ 1;
        dst->unwrap_have[o] = 1;
        dst->unwrap_b[o] = winb[g.nwin - 1];
        dst->unwrap_m[o] = s_m[g.nwin - 1 - w0];
    }
}

cudaError_t launch_demap(const EqParams &p, const EqGeom &g, int resolve_amb, int uw_in, const uint8_t *dec,
                         const uint8_t *winb, float4 *dbg_win, const uint8_t *prbs, uint8_t *bits_out,
                         DevState *dst, cudaStream_t st)
{
    unsigned grid = (unsigned)((g.nwin + kDemapWin - 1) / kDemapWin);
    if (p.kk)
        k_demap<true><<<grid, kDemapThreads, 0, st>>>(p, g, resolve_amb, uw_in, dec, winb, dbg_win, prbs,
                                                      bits_out, dst);
    else
        k_demap<false><<<grid, kDemapThreads, 0, st>>>(p, g, resolve_amb, uw_in, dec, winb, dbg_win, prbs,
                                                       bits_out, dst);
    return cudaGetLastError();
}

}  // namespace rxk
