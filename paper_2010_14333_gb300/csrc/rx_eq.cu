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
//
// Frozen form (QAM only): every window of a block filters with the call's start
// taps, so the filter of the call is one fixed FIR (computed here in FP32, or
// passed in as soft symbols by the tensor-core block-Toeplitz kernel); the warp
// of the last block sums sum_k y[2k+TH-i] conj(e_k) over its windows and writes
// start taps + mu (64 / eq_block) times that sum as the next call's taps.
#include <type_traits>

#include "rx_async.cuh"
#include "rx_common.cuh"
#include "rx_internal.cuh"

namespace rxk {

// ------------------------------------------------------------- symbol helpers
__device__ __forceinline__ int gray(int L) { return L ^ (L >> 1); }
__device__ __forceinline__ int gray_inv(int g)
{
    int L = g;
    for (int s = g >> 1; s; s >>= 1) L ^= s;
    return L;
}
// ---------------------------------------------------------------- one window
// ys: 2-sps input in shared memory (16-byte aligned); c0: local index of y[2 k0]
// (even); the window's 64 symbols are k0..k0+63.  mode: 0 CMA, 1 data-aided (PAM
// training), 2 decision directed.  NT taps, TH = (NT-1)/2 odd, MQ levels per
// dimension: compile-time so that every loop unrolls.
struct WinOut {
    int b;
    float best, second;
    unsigned errA, errB;   // bit errors of the window under absolute rotations 0,1 | 2,3 (16 bits each)
    unsigned serr;         // symbol errors under rotations 0..3 (8 bits each)
    unsigned nnear;        // symbols within 1e-4 of a threshold
};

// reference bit group of BPS bits, MSB first, at PRBS position pos of the
// bit-packed table (bit j at word j>>5, bit 31-(j&31)); the table repeats the
// first 256 bits after the period, so pos + BPS never wraps
template <int BPS>
__device__ __forceinline__ int ref_bits(const uint32_t *__restrict__ tab, int pos)
{
    uint32_t w0 = __ldg(tab + (pos >> 5)), w1 = __ldg(tab + (pos >> 5) + 1);
    return (int)(__funnelshift_l(w1, w0, pos & 31) >> (32 - BPS));
}

// rotate a level-index pair by -j, q times (q in 0..3)
template <int MQ>
__device__ __forceinline__ void rot_t(int &LI, int &LQ, int q)
{
    int a = LI, b = LQ;
    if (q & 2) { a = MQ - 1 - a; b = MQ - 1 - b; }   // times -1
    if (q & 1) { int t = a; a = b; b = MQ - 1 - t; } // times -j
    LI = a;
    LQ = b;
}

template <int MQ>
__device__ __forceinline__ int decide_t(float t)
{
    int L = 0;
#pragma unroll
    for (int j = 0; j < MQ - 1; j++) L += (t >= (float)(2 * j - (MQ - 2)));
    return L;
}
template <int MQ>
__device__ __forceinline__ bool near_t(float t)
{
    bool n = false;
#pragma unroll
    for (int j = 0; j < MQ - 1; j++) n |= fabsf(t - (float)(2 * j - (MQ - 2))) < 1e-4f;
    return n;
}
// squared distance to the nearest level of the odd-integer grid scaled by r: fold |t|
// about the level mid-points (4 levels: (||t| - 2r| - r)^2; 2 levels: (|t| - r)^2)
template <int MQ>
__device__ __forceinline__ float dist_s(float t, float r, float acc)
{
    float a = fabsf(t);
#pragma unroll
    for (int h = MQ >> 1; h > 1; h >>= 1) a = fabsf(a - (float)h * r);
    a -= r;
    return fmaf(a, a, acc);
}

template <int NT, int MQ, bool FRZ = false>
__device__ __forceinline__ WinOut qam_window(const EqParams &p, const float2 *ys, int c0, float2 *zs, float2 *es,
                                             float2 *ws, int mode, float mu, int lane, uint8_t *dec_out,
                                             float2 *dbg_z, const uint32_t *prbs_bits, int pwin,
                                             float2 tph, const float2 *zin = nullptr, float2 *G = nullptr)
{
    constexpr int TH = (NT - 1) / 2;
    constexpr int NP = (NT + 1) / 2;              // y pairs per symbol
    static_assert(TH % 2 == 1, "tap half-length must be odd");
    // filter: z_k = sum_i conj(w_i) y[2k + TH - i]; pairs start at the even index 2k - TH - 1.
    // The tap pair (w[NT-1-2v], w[NT-2v]) is one 16-byte shared-memory broadcast
    // (ws holds NT+1 entries, the last one zero), shared by the lane's two symbols.
    if (FRZ && zin) {   // soft symbols from the block-Toeplitz kernel
#pragma unroll
        for (int h = 0; h < 2; h++) {
            int q = lane + 32 * h;
            float2 zq = zin[q];
            zs[q] = zq;
            if (dbg_z) dbg_z[q] = zq;
        }
    } else {
        const float4 *yp0 = reinterpret_cast<const float4 *>(ys + c0 + 2 * lane - TH - 1);
        const float4 *yp1 = reinterpret_cast<const float4 *>(ys + c0 + 2 * (lane + 32) - TH - 1);
        const float4 *wp = reinterpret_cast<const float4 *>(ws);
        float ar0 = 0.f, ai0 = 0.f, ar1 = 0.f, ai1 = 0.f;
#pragma unroll
        for (int v = 0; v < NP; v++) {
            const float4 W = wp[(NT - 1 - 2 * v) / 2];
            const float4 Y0 = yp0[v], Y1 = yp1[v];
            // offset 2v+1 -> tap NT-1-2v
            ar0 = fmaf(W.x, Y0.z, fmaf(W.y, Y0.w, ar0));
            ai0 = fmaf(W.x, Y0.w, fmaf(-W.y, Y0.z, ai0));
            ar1 = fmaf(W.x, Y1.z, fmaf(W.y, Y1.w, ar1));
            ai1 = fmaf(W.x, Y1.w, fmaf(-W.y, Y1.z, ai1));
            if (v >= 1) {   // offset 2v -> tap NT-2v
                ar0 = fmaf(W.z, Y0.x, fmaf(W.w, Y0.y, ar0));
                ai0 = fmaf(W.z, Y0.y, fmaf(-W.w, Y0.x, ai0));
                ar1 = fmaf(W.z, Y1.x, fmaf(W.w, Y1.y, ar1));
                ai1 = fmaf(W.z, Y1.y, fmaf(-W.w, Y1.x, ai1));
            }
        }
        zs[lane] = make_float2(ar0, ai0);
        zs[lane + 32] = make_float2(ar1, ai1);
        if (dbg_z) {
            dbg_z[lane] = make_float2(ar0, ai0);
            dbg_z[lane + 32] = make_float2(ar1, ai1);
        }
    }
    __syncwarp();
    WinOut R;
    R.b = -1;
    R.best = 0.f;
    R.second = 0.f;
    float cs = 1.f, sn = 0.f;   // cos / sin of the chosen phase
    if (mode == 2) {
        // blind phase search: lane b tests theta_b = (b/B)(pi/2) - pi/4 (tph = cos, sin).
        // The rotated, scaled symbol s z e^{-j theta} divided by s cos(theta) is
        // (zr + zi tan, zi - zr tan): one FMA per dimension.  Its distance to the
        // nearest level is that of the original with the level grid scaled by
        // 1 / (s cos), times (s cos)^2, a factor common to the whole window.
        const float tcs = tph.x, tsn = tph.y;
        const float tn = tsn / tcs, sc = p.scale * tcs, r = 1.f / sc;
        float M = 0.f;
        const float4 *z4 = reinterpret_cast<const float4 *>(zs);
#pragma unroll 8
        for (int q2 = 0; q2 < kWin / 2; q2++) {
            float4 Z = z4[q2];
            M = dist_s<MQ>(fmaf(Z.y, tn, Z.x), r, M);
            M = dist_s<MQ>(fmaf(-Z.x, tn, Z.y), r, M);
            M = dist_s<MQ>(fmaf(Z.w, tn, Z.z), r, M);
            M = dist_s<MQ>(fmaf(-Z.z, tn, Z.w), r, M);
        }
        M *= sc * sc;
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
    constexpr int NB = MQ == 2 ? 1 : 2, BPS = 2 * NB;
    unsigned eA = 0, eB = 0, se = 0, nn = 0;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        int q = lane + 32 * h;
        float2 z = zs[q];
        float vr = p.scale * fmaf(z.x, cs, z.y * sn);
        float vi = p.scale * fmaf(z.y, cs, -z.x * sn);
        int LI = decide_t<MQ>(vr), LQ = decide_t<MQ>(vi);
        bool nr = near_t<MQ>(vr) || near_t<MQ>(vi);
        if (dec_out) dec_out[q] = (uint8_t)(LI | (LQ << 3) | (nr ? 64 : 0));
        if (prbs_bits) {
            // bit errors of this symbol under each absolute pi/2 rotation of the decision
            // with gray(MQ-1-L) = gray(L) ^ cm, rotation q of (LI, LQ) has the code
            // q0: (gI, gQ), q1: (gQ, gI^cm), q2: (gI^cm, gQ^cm), q3: (gQ^cm, gI)
            const int ref = ref_bits<BPS>(prbs_bits, pwin + BPS * q);
            constexpr int cm = MQ == 2 ? 1 : 2;
            const int gI = gray(LI), gQ = gray(LQ);
            const int X = ((gI << NB) | gQ) ^ ref, Xs = ((gQ << NB) | gI) ^ ref;
            const unsigned n0 = __popc(X), n1 = __popc(Xs ^ cm), n2 = __popc(X ^ ((cm << NB) | cm)),
                           n3 = __popc(Xs ^ (cm << NB));
            eA += n0 + (n1 << 16);
            eB += n2 + (n3 << 16);
            se += (unsigned)(n0 > 0) | ((unsigned)(n1 > 0) << 8) | ((unsigned)(n2 > 0) << 16) |
                  ((unsigned)(n3 > 0) << 24);
            nn += nr;
        }
        float2 e;
        if (mode == 0) {
            float f = p.r2 - (z.x * z.x + z.y * z.y);
            e = make_float2(z.x * f, z.y * f);
        } else {
            float dI = (float)(2 * LI - (MQ - 1)) * inv_s, dQ = (float)(2 * LQ - (MQ - 1)) * inv_s;
            e = make_float2(fmaf(dI, cs, -dQ * sn) - z.x, fmaf(dI, sn, dQ * cs) - z.y);
        }
        es[q] = e;
    }
    __syncwarp();
    if (prbs_bits) {
        R.errA = warp_sum_i(eA);
        R.errB = warp_sum_i(eB);
        R.serr = warp_sum_i(se);
        R.nnear = warp_sum_i(nn);
    }
    // block-LMS update after the window: w_i += mu sum_k y[2k + TH - i] conj(e_k);
    // frozen form: the sum only, accumulated in G (last block), taps unchanged
    if (lane < NT && (!FRZ || G)) {
        float gr = 0.f, gi = 0.f;
        const float2 *yb = ys + (c0 + TH - lane);
        const float4 *e4 = reinterpret_cast<const float4 *>(es);
#pragma unroll 8
        for (int q2 = 0; q2 < kWin / 2; q2++) {
            float4 E = e4[q2];
            float2 y0 = yb[4 * q2], y1 = yb[4 * q2 + 2];
            gr = fmaf(y0.x, E.x, fmaf(y0.y, E.y, gr));
            gi = fmaf(y0.y, E.x, fmaf(-y0.x, E.y, gi));
            gr = fmaf(y1.x, E.z, fmaf(y1.y, E.w, gr));
            gi = fmaf(y1.y, E.z, fmaf(-y1.x, E.w, gi));
        }
        if (FRZ) {
            G->x += gr;
            G->y += gi;
        } else {
            float2 wl = ws[lane];
            ws[lane] = make_float2(fmaf(mu, gr, wl.x), fmaf(mu, gi, wl.y));
        }
    }
    __syncwarp();
    return R;
}

template <int NT, int MQ>
__device__ __forceinline__ WinOut pam_window(const EqParams &p, const float *ys, int c0, long long k0, float *zs,
                                             float *es, float *ws, int mode, float mu, int lane, uint8_t *dec_out,
                                             float2 *dbg_z, const uint8_t *prbs_ext, const uint32_t *prbs_bits,
                                             int pwin)
{
    WinOut R;
    R.b = 0;
    R.best = R.second = 0.f;
    R.errA = R.errB = R.serr = R.nnear = 0;
    unsigned e0 = 0, s0 = 0, nn = 0;
    constexpr int TH = (NT - 1) / 2;
    constexpr int NP = (NT + 1) / 2;
    static_assert(TH % 2 == 1, "tap half-length must be odd");
    float w[2 * NP];
#pragma unroll
    for (int i = 0; i < NP; i++) {
        float2 t = reinterpret_cast<const float2 *>(ws)[i];
        w[2 * i] = t.x;
        w[2 * i + 1] = t.y;
    }
    constexpr int nb = MQ == 2 ? 1 : (MQ == 4 ? 2 : 3);
    long long pb = (mode == 1) ? (long long)(((long long)nb * k0) % 32767) : 0;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        int q = lane + 32 * h;
        const float2 *yp = reinterpret_cast<const float2 *>(ys + c0 + 2 * q - TH - 1);
        float a = 0.f;
#pragma unroll
        for (int v = 0; v < NP; v++) {
            float2 Y = yp[v];
            a = fmaf(w[NT - 1 - 2 * v], Y.y, a);
            if (v >= 1) a = fmaf(w[NT - 2 * v], Y.x, a);
        }
        zs[q] = a;
        if (dbg_z) dbg_z[q] = make_float2(a, 0.f);
        int L = decide_t<MQ>(a);
        bool nr = near_t<MQ>(a);
        if (dec_out) dec_out[q] = (uint8_t)(L | (nr ? 64 : 0));
        if (prbs_bits) {
            unsigned ne = __popc(gray(L) ^ ref_bits<nb>(prbs_bits, pwin + nb * q));
            e0 += ne;
            s0 += ne > 0;
            nn += nr;
        }
        float d;
        if (mode == 1) {   // data aided: the transmitted level from the PRBS
            int pos = (int)(pb + nb * q);
            pos = pos >= 32767 ? pos - 32767 : pos;
            int gi = 0;
            for (int t = 0; t < nb; t++) gi = (gi << 1) | prbs_ext[pos + t];
            d = (float)(2 * gray_inv(gi) - (MQ - 1));
        } else {
            d = (float)(2 * L - (MQ - 1));
        }
        es[q] = d - a;
    }
    __syncwarp();
    if (prbs_bits) {
        R.errA = warp_sum_i(e0);
        R.serr = warp_sum_i(s0);
        R.nnear = warp_sum_i(nn);
    }
    if (lane < NT) {
        const float *yb = ys + (c0 + TH - lane);
        float g = 0.f;
#pragma unroll 16
        for (int q = 0; q < kWin; q++) g = fmaf(yb[2 * q], es[q], g);
        ws[lane] = fmaf(mu, g, ws[lane]);
    }
    __syncwarp();
    return R;
}

// cos and sin of the test phase of this lane, theta_b = (b/B)(pi/2) - pi/4
__device__ __forceinline__ float2 test_phase(const EqParams &p, int lane)
{
    float sn, cs;
    sincospif((float)lane / (float)(2 * p.bps_b) - 0.25f, &sn, &cs);
    return make_float2(cs, sn);
}

// -------------------------------------------------------------- equaliser kernel
// Payload: one warp per block of eq_block symbols, input staged by one bulk copy.
// Training (train=1): one warp runs the training windows sequentially, staging
// each window's input with plain loads.
template <bool QAM, int NT, int MQ>
__global__ void __launch_bounds__(32 * kEqWarpsMax)
    k_eq(EqParams p, EqGeom g, int train, const void *__restrict__ Yv, float2 *taps_in, float2 *taps_out,
         uint8_t *__restrict__ dec, uint8_t *__restrict__ winb, uint4 *__restrict__ winrec,
         float4 *__restrict__ dbg_win, float2 *__restrict__ dbg_z, const uint8_t *__restrict__ prbs_ext,
         const uint32_t *__restrict__ prbs_bits, DevState *dst)
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
    long long blk = (long long)blockIdx.x * (blockDim.x >> 5) + wid;
    if (!train && blk >= g.nblk) return;
    // start taps; the slot past the last tap stays zero for the paired loads
    if (QAM) reinterpret_cast<float2 *>(ws)[lane] = lane < NT ? taps_in[lane] : make_float2(0.f, 0.f);
    else reinterpret_cast<float *>(ws)[lane] = lane < NT ? taps_in[lane].x : 0.f;
    __syncwarp();
    unsigned ambig = 0;
    const float2 tph = test_phase(p, lane);
    if (train) {
        for (long long k0 = 0; k0 < p.ntrain; k0 += kWin) {
            long long ym0 = 2 * k0 - kYHist;
            for (int i = lane; i < ylen; i += 32) ys[i] = Y[ym0 + i - g.ybase];
            __syncwarp();
            float2 *dz = dbg_z ? dbg_z + (k0 - g.sym_lo) : nullptr;
            if (QAM) {
                int mode = (k0 < p.ncma) ? 0 : 2;
                float mu = mode == 0 ? p.mu_cma : p.mu;
                qam_window<NT, MQ>(p, reinterpret_cast<float2 *>(ys), kYHist, reinterpret_cast<float2 *>(zs),
                                   reinterpret_cast<float2 *>(es), reinterpret_cast<float2 *>(ws), mode, mu, lane,
                                   nullptr, dz, nullptr, 0, tph);
            } else {
                pam_window<NT, MQ>(p, reinterpret_cast<float *>(ys), kYHist, k0, reinterpret_cast<float *>(zs),
                                   reinterpret_cast<float *>(es), reinterpret_cast<float *>(ws), 1, p.mu_train, lane,
                                   nullptr, dz, prbs_ext, nullptr, 0);
            }
        }
        if (lane < NT)
            taps_in[lane] = QAM ? reinterpret_cast<float2 *>(ws)[lane]
                                : make_float2(reinterpret_cast<float *>(ws)[lane], 0.f);
        return;
    }
    long long kb = g.pay_lo + blk * B;
    long long ym0 = 2 * kb - kYHist;
    const bool last = blk == g.nblk - 1;
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
    const int bpsv = p.bps;
    int pwin = (int)(((long long)bpsv * kb) % 32767);   // PRBS position of the window's first bit
    for (int w = 0; w < B / kWin; w++) {
        long long k0 = kb + (long long)w * kWin;
        int c0 = kYHist + 2 * w * kWin;
        uint8_t *dq = dec + (k0 - g.pay_lo);
        float2 *dz = dbg_z ? dbg_z + (k0 - g.sym_lo) : nullptr;
        long long wi = (k0 - g.pay_lo) / kWin;
        if (QAM) {
            WinOut R = qam_window<NT, MQ>(p, reinterpret_cast<float2 *>(ys), c0, reinterpret_cast<float2 *>(zs),
                                          reinterpret_cast<float2 *>(es), reinterpret_cast<float2 *>(ws), 2, p.mu,
                                          lane, dq, dz, prbs_bits, pwin, tph);
            if (lane == 0) {
                winb[wi] = (uint8_t)R.b;
                winrec[wi] = make_uint4(R.errA, R.errB, R.serr, (unsigned)R.b | (R.nnear << 8));
                if (dbg_win) dbg_win[wi] = make_float4((float)R.b, 0.f, R.best, R.second);
                ambig += (R.second - R.best) <= 1e-6f * R.best;
            }
        } else {
            WinOut R = pam_window<NT, MQ>(p, reinterpret_cast<float *>(ys), c0, k0, reinterpret_cast<float *>(zs),
                                          reinterpret_cast<float *>(es), reinterpret_cast<float *>(ws), 2, p.mu, lane,
                                          dq, dz, prbs_ext, prbs_bits, pwin);
            if (lane == 0) {
                winb[wi] = 0;
                winrec[wi] = make_uint4(R.errA, 0u, R.serr, R.nnear << 8);
            }
        }
        pwin += bpsv * kWin;
        pwin = pwin >= 32767 ? pwin - 32767 : pwin;
    }
    if (last && lane < NT) {
        taps_out[lane] = QAM ? reinterpret_cast<float2 *>(ws)[lane]
                             : make_float2(reinterpret_cast<float *>(ws)[lane], 0.f);
    }
    if (lane == 0 && ambig) atomicAdd(&dst->cnt[C_AMBIG], (unsigned long long)ambig);
}

// ------------------------------------------------- frozen form, window-parallel
// Every payload block filters with the call's start taps, so no window depends
// on another: one warp per 64-symbol window.  With soft symbols from the
// block-Toeplitz kernel (zin) only the windows of the last block read the
// input, for the tap step; without, each window stages its input and filters
// on the CUDA cores.  The last block's windows leave their partial sums of
// y conj(e) in gpart; the warp that finishes last (ticket) adds them in window
// order, so the next taps do not depend on the order the warps ran in.
template <int NT, int MQ>
__global__ void __launch_bounds__(32 * kEqWarpsMax)
    k_eq_frozen(EqParams p, EqGeom g, const float2 *__restrict__ Y, const float2 *__restrict__ zin,
                const float2 *__restrict__ taps_in, float2 *__restrict__ taps_out, uint8_t *__restrict__ dec,
                uint8_t *__restrict__ winb, uint4 *__restrict__ winrec, float4 *__restrict__ dbg_win,
                float2 *__restrict__ dbg_z, const uint32_t *__restrict__ prbs_bits, DevState *dst)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int ylen = 2 * kWin + 2 * kYHist;
    constexpr size_t per_warp = (16 + (size_t)(ylen + 2 * kWin + 32) * sizeof(float2) + 15) & ~(size_t)15;
    unsigned char *base = smraw + per_warp * wid;
    uint64_t *bar = reinterpret_cast<uint64_t *>(base);
    float2 *ys = reinterpret_cast<float2 *>(base + 16);
    float2 *zs = ys + ylen;
    float2 *es = zs + kWin;
    float2 *ws = es + kWin;
    const long long wi = (long long)blockIdx.x * (blockDim.x >> 5) + wid;
    if (wi >= g.nwin) return;
    const int nlast = p.eq_block / kWin;            // windows of the last block
    const long long wl = (long long)g.nwin - nlast;  // its first window
    const bool last = wi >= wl;
    ws[lane] = lane < NT ? taps_in[lane] : make_float2(0.f, 0.f);
    __syncwarp();
    const long long k0 = g.pay_lo + wi * kWin;
    if (!zin || last) {
        if (lane == 0) {
            mbar_init(bar, 1);
            mbar_expect_tx(bar, (unsigned)(ylen * sizeof(float2)));
            bulk_g2s(ys, Y + (2 * k0 - kYHist - g.ybase), (unsigned)(ylen * sizeof(float2)), bar);
        }
        __syncwarp();
        if (!mbar_wait(bar, 0)) {
            if (lane == 0) atomicExch(&dst->err, (int)RX_ETIMEOUT);
            mbar_wait(bar, 0);
            return;
        }
    }
    const int pwin = (int)(((long long)p.bps * k0) % 32767);
    float2 G = make_float2(0.f, 0.f);
    WinOut R = qam_window<NT, MQ, true>(p, ys, kYHist, zs, es, ws, 2, p.mu, lane, dec + (k0 - g.pay_lo),
                                        dbg_z ? dbg_z + (k0 - g.sym_lo) : nullptr, prbs_bits, pwin,
                                        test_phase(p, lane), zin ? zin + (k0 - g.pay_lo) : nullptr,
                                        last ? &G : nullptr);
    const long long wq = (k0 - g.pay_lo) / kWin;
    if (lane == 0) {
        winb[wq] = (uint8_t)R.b;
        winrec[wq] = make_uint4(R.errA, R.errB, R.serr, (unsigned)R.b | (R.nnear << 8));
        if (dbg_win) dbg_win[wq] = make_float4((float)R.b, 0.f, R.best, R.second);
        if ((R.second - R.best) <= 1e-6f * R.best) atomicAdd(&dst->cnt[C_AMBIG], 1ull);
    }
    if (!last) return;
    float2 *gp = g.gpart + (wi - wl) * 32;
    if (lane < NT) gp[lane] = G;
    __threadfence();
    __syncwarp();
    unsigned t = 0;
    if (lane == 0) t = atomicAdd(&dst->eq_ticket, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t != (unsigned)nlast - 1) return;
    __threadfence();
    if (lane < NT) {
        float gr = 0.f, gi = 0.f;
        for (int j = 0; j < nlast; j++) {
            float2 v = __ldcg(g.gpart + j * 32 + lane);
            gr += v.x;
            gi += v.y;
        }
        const float step = p.mu * (float)kWin / (float)p.eq_block;
        float2 w0 = ws[lane];
        taps_out[lane] = make_float2(fmaf(step, gr, w0.x), fmaf(step, gi, w0.y));
    }
    if (lane == 0) dst->eq_ticket = 0;
}

static size_t eq_smem_frozen_per_warp()
{
    return (16 + (size_t)(2 * kWin + 2 * kYHist + 2 * kWin + 32) * sizeof(float2) + 15) & ~(size_t)15;
}

static size_t eq_smem_per_warp(bool qam, int B)
{
    size_t el = qam ? sizeof(float2) : sizeof(float);
    size_t w = 16 + (size_t)(2 * B + 2 * kYHist + 2 * kWin + 32) * el;
    return (w + 15) & ~(size_t)15;
}

template <bool QAM, int NT, int MQ>
static cudaError_t launch_eq_t(const EqParams &p, const EqGeom &g, int train, const void *Y, const float2 *zin,
                               float2 *taps_in, float2 *taps_out, uint8_t *dec, uint8_t *winb, uint4 *winrec,
                               float4 *dbg_win, float2 *dbg_z, const uint8_t *prbs, const uint32_t *prbs_bits,
                               DevState *dst, cudaStream_t st)
{
    if (train) {
        size_t smem = eq_smem_per_warp(QAM, kWin);
        k_eq<QAM, NT, MQ><<<1, 32, smem, st>>>(p, g, 1, Y, taps_in, taps_out, dec, winb, winrec, dbg_win, dbg_z,
                                               prbs, prbs_bits, dst);
        return cudaGetLastError();
    }
    if constexpr (QAM) {
        if (p.frozen) {
            if (g.nwin < p.eq_block / kWin) return cudaErrorInvalidValue;
            // every call counts its last block's windows from zero, whatever an earlier
            // launch that gave up on a bounded wait left in the ticket
            cudaError_t e = cudaMemsetAsync(&dst->eq_ticket, 0, sizeof(unsigned), st);
            if (e != cudaSuccess) return e;
            unsigned grid = (unsigned)((g.nwin + p.warps - 1) / p.warps);
            k_eq_frozen<NT, MQ><<<grid, 32 * p.warps, eq_smem_frozen_per_warp() * p.warps, st>>>(
                p, g, (const float2 *)Y, zin, taps_in, taps_out, dec, winb, winrec, dbg_win, dbg_z, prbs_bits, dst);
            return cudaGetLastError();
        }
    }
    size_t smem = eq_smem_per_warp(QAM, p.eq_block) * p.warps;
    unsigned grid = (unsigned)((g.nblk + p.warps - 1) / p.warps);
    k_eq<QAM, NT, MQ><<<grid, 32 * p.warps, smem, st>>>(p, g, 0, Y, taps_in, taps_out, dec, winb, winrec, dbg_win,
                                                          dbg_z, prbs, prbs_bits, dst);
    return cudaGetLastError();
}

// shared-memory attribute of the payload kernel, set to the largest CTA any
// handle may launch (the attribute belongs to the function, which handles with
// different CTA shapes share); set at handle creation so that launches (and graph
// captures) make no attribute calls
template <bool QAM, int NT, int MQ>
static cudaError_t prepare_eq_t(const EqParams &p)
{
    const int smem = (int)kMaxSmemCta;
    if constexpr (QAM) {
        if (p.frozen)
            return cudaFuncSetAttribute(k_eq_frozen<NT, MQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }
    return cudaFuncSetAttribute(k_eq<QAM, NT, MQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// ----------------------------------- symbol-by-symbol DD-LMS (KK, eq_mode 1)
// The paper's short KK equaliser (Sec. 2, KK chain): a decision-directed LMS
// whose complex taps are updated after every symbol, so that they follow the
// clock phase and the symbol phase together; no phase search.  One thread runs
// one block's recursion (the training: one thread over the training symbols,
// CMA for the first ncma):
//   z_k = sum_j conj(w_j) y[2k + TH - j],  decision on s z_k,
//   e = z (R2 - |z|^2) (CMA) or d / s - z (decision directed),
//   w_j += mu y[2k + TH - j] conj(e).
// The inputs of the next symbol are those of this one moved by two samples.
constexpr int kDdU = 8;   // symbols per batch of loaded samples

template <int NT, int MQ>
__global__ void __launch_bounds__(128)
    k_eq_dd(EqParams p, EqGeom g, int train, const float2 *__restrict__ Y, float2 *taps_in, float2 *taps_out,
            uint8_t *__restrict__ dec, float2 *__restrict__ dbg_z)
{
    constexpr int TH = (NT - 1) / 2;
    const long long blk = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (train ? blk > 0 : blk >= g.nblk) return;
    float2 w[NT];
#pragma unroll
    for (int j = 0; j < NT; j++) w[j] = taps_in[j];
    const long long k0 = train ? 0 : g.pay_lo + blk * p.eq_block;
    const long long n = train ? p.ntrain : p.eq_block;
    const long long cma_until = train ? p.ncma : -1;
    const float s = p.scale, inv_s = 1.0f / p.scale;
    float2 yv[NT];   // yv[j] = y[2k + TH - j]
#pragma unroll
    for (int j = 0; j < NT; j++) yv[j] = Y[2 * k0 + TH - j - g.ybase];
    // the samples that enter the window, kDdU symbols at a time: batch b brings
    // y[2 kb + TH + 1 + i], i < 2 kDdU (kb its first symbol), loaded while the batch
    // before it is computed (n is a multiple of kDdU; the last batch reads two samples
    // past the last symbol's window, inside the workspace, and never uses them)
    float2 nx[2 * kDdU];
#pragma unroll
    for (int i = 0; i < 2 * kDdU; i++) nx[i] = Y[2 * k0 + TH + 1 + i - g.ybase];
    for (long long q0 = 0; q0 < n; q0 += kDdU) {
        float2 cb[2 * kDdU];
#pragma unroll
        for (int i = 0; i < 2 * kDdU; i++) cb[i] = nx[i];
        if (q0 + kDdU < n) {
#pragma unroll
            for (int i = 0; i < 2 * kDdU; i++) nx[i] = Y[2 * (k0 + q0 + kDdU) + TH + 1 + i - g.ybase];
        }
#pragma unroll
        for (int u = 0; u < kDdU; u++) {
            const long long k = k0 + q0 + u;
            float zr = 0.f, zi = 0.f;
#pragma unroll
            for (int j = 0; j < NT; j++) {   // conj(w) y
                zr = fmaf(w[j].x, yv[j].x, fmaf(w[j].y, yv[j].y, zr));
                zi = fmaf(w[j].x, yv[j].y, fmaf(-w[j].y, yv[j].x, zi));
            }
            const float vr = s * zr, vi = s * zi;
            const int LI = decide_t<MQ>(vr), LQ = decide_t<MQ>(vi);
            const bool nr = near_t<MQ>(vr) || near_t<MQ>(vi);
            if (!train) dec[k - g.pay_lo] = (uint8_t)(LI | (LQ << 3) | (nr ? 64 : 0));
            if (dbg_z) dbg_z[k - g.sym_lo] = make_float2(zr, zi);
            float er, ei, mu;
            if (k < cma_until) {
                const float f = p.r2 - (zr * zr + zi * zi);
                er = zr * f;
                ei = zi * f;
                mu = p.mu_cma;
            } else {
                er = (float)(2 * LI - (MQ - 1)) * inv_s - zr;
                ei = (float)(2 * LQ - (MQ - 1)) * inv_s - zi;
                mu = p.mu;
            }
#pragma unroll
            for (int j = 0; j < NT; j++) {   // w += mu y conj(e)
                w[j].x = fmaf(mu, fmaf(yv[j].x, er, yv[j].y * ei), w[j].x);
                w[j].y = fmaf(mu, fmaf(yv[j].y, er, -yv[j].x * ei), w[j].y);
            }
#pragma unroll
            for (int j = NT - 1; j >= 2; j--) yv[j] = yv[j - 2];
            yv[1] = cb[2 * u];
            yv[0] = cb[2 * u + 1];
        }
    }
    if (train) {
#pragma unroll
        for (int j = 0; j < NT; j++) taps_in[j] = w[j];
    } else if (blk == g.nblk - 1) {
#pragma unroll
        for (int j = 0; j < NT; j++) taps_out[j] = w[j];
    }
}

// window records of the symbol-by-symbol form: one warp per 64-symbol window, from
// the decisions: bit errors under the four absolute pi/2 rotations (as the window
// equaliser scores them), near-threshold count, phase index 0
template <int MQ>
__global__ void __launch_bounds__(128)
    k_dd_score(EqParams p, EqGeom g, const uint8_t *__restrict__ dec, uint8_t *__restrict__ winb,
               uint4 *__restrict__ winrec, float4 *__restrict__ dbg_win, const uint32_t *__restrict__ prbs_bits)
{
    constexpr int NB = MQ == 2 ? 1 : 2, BPS = 2 * NB;
    const int lane = threadIdx.x & 31;
    const long long wi = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wi >= g.nwin) return;
    const long long k0 = g.pay_lo + wi * kWin;
    const int pwin = (int)(((long long)BPS * k0) % 32767);
    unsigned eA = 0, eB = 0, se = 0, nn = 0;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int q = lane + 32 * h;
        const int d = dec[wi * kWin + q];
        const int LI = d & 7, LQ = (d >> 3) & 7;
        const int ref = ref_bits<BPS>(prbs_bits, pwin + BPS * q);
        constexpr int cm = MQ == 2 ? 1 : 2;
        const int gI = gray(LI), gQ = gray(LQ);
        const int X = ((gI << NB) | gQ) ^ ref, Xs = ((gQ << NB) | gI) ^ ref;
        const unsigned n0 = __popc(X), n1 = __popc(Xs ^ cm), n2 = __popc(X ^ ((cm << NB) | cm)),
                       n3 = __popc(Xs ^ (cm << NB));
        eA += n0 + (n1 << 16);
        eB += n2 + (n3 << 16);
        se += (unsigned)(n0 > 0) | ((unsigned)(n1 > 0) << 8) | ((unsigned)(n2 > 0) << 16) | ((unsigned)(n3 > 0) << 24);
        nn += (d & 64) != 0;
    }
    eA = warp_sum_i(eA);
    eB = warp_sum_i(eB);
    se = warp_sum_i(se);
    nn = warp_sum_i(nn);
    if (lane == 0) {
        winb[wi] = 0;
        winrec[wi] = make_uint4(eA, eB, se, nn << 8);
        if (dbg_win) dbg_win[wi] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <int NT, int MQ>
static cudaError_t launch_eq_dd(const EqParams &p, const EqGeom &g, int train, const float2 *Y, float2 *taps_in,
                                float2 *taps_out, uint8_t *dec, uint8_t *winb, uint4 *winrec, float4 *dbg_win,
                                float2 *dbg_z, const uint32_t *prbs_bits, cudaStream_t st)
{
    if (train) {
        k_eq_dd<NT, MQ><<<1, 32, 0, st>>>(p, g, 1, Y, taps_in, taps_out, dec, dbg_z);
        return cudaGetLastError();
    }
    k_eq_dd<NT, MQ><<<(unsigned)((g.nblk + 127) / 128), 128, 0, st>>>(p, g, 0, Y, taps_in, taps_out, dec, dbg_z);
    if (g.nwin > 0)
        k_dd_score<MQ><<<(unsigned)((g.nwin + 3) / 4), 128, 0, st>>>(p, g, dec, winb, winrec, dbg_win, prbs_bits);
    return cudaGetLastError();
}

// tap counts with a compiled kernel (odd, half-length odd)
#define RX_EQ_TAPS(X) X(3) X(7) X(11) X(15) X(19) X(23) X(27) X(31)

size_t eq_smem_bytes(const EqParams &p, int warps) { return eq_smem_per_warp(p.kk != 0, p.eq_block) * warps; }

cudaError_t prepare_eq(const EqParams &p)
{
    if (p.dd) return cudaSuccess;   // the symbol-by-symbol kernels take no dynamic shared memory
#define RX_PREP(NTV)                                                                                           \
    if (p.ntaps == NTV) {                                                                                      \
        if (p.kk && p.mq == 2) return prepare_eq_t<true, NTV, 2>(p);                                            \
        if (p.kk && p.mq == 4) return prepare_eq_t<true, NTV, 4>(p);                                            \
        if (!p.kk && p.mq == 2) return prepare_eq_t<false, NTV, 2>(p);                                          \
        if (!p.kk && p.mq == 4) return prepare_eq_t<false, NTV, 4>(p);                                          \
        if (!p.kk && p.mq == 8) return prepare_eq_t<false, NTV, 8>(p);                                          \
    }
    RX_EQ_TAPS(RX_PREP)
#undef RX_PREP
    return cudaErrorInvalidValue;
}

cudaError_t launch_eq(const EqParams &p, const EqGeom &g, int train, const void *Y, const float2 *zin,
                      float2 *taps_in, float2 *taps_out, uint8_t *dec, uint8_t *winb, uint4 *winrec, float4 *dbg_win,
                      float2 *dbg_z, const uint8_t *prbs, const uint32_t *prbs_bits, DevState *dst, cudaStream_t st)
{
    if (p.dd) {
        const float2 *Yc = (const float2 *)Y;
#define RX_DD(NTV)                                                                                             \
        if (p.ntaps == NTV && p.mq == 4)                                                                       \
            return launch_eq_dd<NTV, 4>(p, g, train, Yc, taps_in, taps_out, dec, winb, winrec, dbg_win, dbg_z,  \
                                        prbs_bits, st);                                                        \
        if (p.ntaps == NTV && p.mq == 2)                                                                       \
            return launch_eq_dd<NTV, 2>(p, g, train, Yc, taps_in, taps_out, dec, winb, winrec, dbg_win, dbg_z,  \
                                        prbs_bits, st);
        RX_DD(2) RX_DD(3) RX_DD(4) RX_DD(5) RX_DD(6) RX_DD(7) RX_DD(8)
#undef RX_DD
        return cudaErrorInvalidValue;
    }
#define RX_CASE(NTV)                                                                                           \
    if (p.ntaps == NTV) {                                                                                      \
        if (p.kk && p.mq == 2) return launch_eq_t<true, NTV, 2>(p, g, train, Y, zin, taps_in, taps_out, dec, winb,  \
                                                                winrec, dbg_win, dbg_z, prbs, prbs_bits, dst, st);                \
        if (p.kk && p.mq == 4) return launch_eq_t<true, NTV, 4>(p, g, train, Y, zin, taps_in, taps_out, dec, winb,  \
                                                                winrec, dbg_win, dbg_z, prbs, prbs_bits, dst, st);                \
        if (!p.kk && p.mq == 2) return launch_eq_t<false, NTV, 2>(p, g, train, Y, zin, taps_in, taps_out, dec,      \
                                                                  winb, winrec, dbg_win, dbg_z, prbs, prbs_bits, dst, st);        \
        if (!p.kk && p.mq == 4) return launch_eq_t<false, NTV, 4>(p, g, train, Y, zin, taps_in, taps_out, dec,      \
                                                                  winb, winrec, dbg_win, dbg_z, prbs, prbs_bits, dst, st);        \
        if (!p.kk && p.mq == 8) return launch_eq_t<false, NTV, 8>(p, g, train, Y, zin, taps_in, taps_out, dec,      \
                                                                  winb, winrec, dbg_win, dbg_z, prbs, prbs_bits, dst, st);        \
    }
    RX_EQ_TAPS(RX_CASE)
#undef RX_CASE
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ demap / BER
// kDemapWin windows per CTA, kDemapWin / 8 per warp.  The pi/2 unwrap
// counter of window w is the carried value plus a prefix sum of integer
// increments; each CTA sums the increments of all earlier windows itself
// (16-byte loads of the window phase indices), then scans its own.  The
// equaliser has already scored every window against the PRBS under the four
// absolute rotations of its decisions (window records), so the bit-error
// statistics here are selections: the decoded rotation q = m + r gives the raw
// count, and the slip-tolerant count takes the best rotation, ties to q.
constexpr int kDemapWin = 32;
constexpr int kDemapThreads = 256;

__device__ __forceinline__ int unwrap_inc(int b_prev, int b, int B)
{
    int d = b_prev - b;
    return (d > B / 2) - (d < -B / 2);
}
__device__ __forceinline__ unsigned rec_err(const uint4 &r, int q)
{
    unsigned v = (q < 2) ? r.x : r.y;
    return (v >> (16 * (q & 1))) & 0xFFFFu;
}
__device__ __forceinline__ unsigned rec_serr(const uint4 &r, int q) { return (r.z >> (8 * q)) & 0xFFu; }

// differential coding: quadrant of a (rotated) decided point (0: I > 0, Q > 0, then
// counterclockwise) and the bits of the point turned back into the first quadrant,
// (1 + 2 b2, 1 + 2 b3) -> lb = b2 b3 (16QAM; QPSK has none)
template <int MQ>
__device__ __forceinline__ int quad_t(int LI, int LQ, int &lb)
{
    const int I = 2 * LI - (MQ - 1), Q = 2 * LQ - (MQ - 1);
    int q, x, y;
    if (I > 0 && Q > 0) { q = 0; x = I; y = Q; }
    else if (I < 0 && Q > 0) { q = 1; x = Q; y = -I; }
    else if (I < 0 && Q < 0) { q = 2; x = -I; y = -Q; }
    else { q = 3; x = -Q; y = I; }
    lb = (MQ == 4) ? ((((x - 1) >> 1) << 1) | ((y - 1) >> 1)) : 0;
    return q;
}

template <bool QAM, int BPS, int MQ>
__global__ void __launch_bounds__(kDemapThreads)
    k_demap(EqParams p, EqGeom g, int resolve_amb, int uw_in, const uint8_t *__restrict__ dec,
            const uint8_t *__restrict__ winb, const uint4 *__restrict__ winrec, float4 *__restrict__ dbg_win,
            uint8_t *__restrict__ bits_out, const uint32_t *__restrict__ prbs_bits, DevState *dst)
{
    constexpr int NW = kDemapThreads / 32;
    constexpr int WPW = kDemapWin / NW;                            // windows per warp
    constexpr int NB = QAM ? BPS / 2 : BPS;
    constexpr int NBYTES = 8 * BPS;                                // 64 symbols * BPS bits / 8
    constexpr int NS = (8 % BPS == 0) ? 8 / BPS : 8 / BPS + 2;     // symbols one output byte touches
    static_assert(kDemapWin == 32 && WPW <= 32, "one scan lane per window of the CTA");
    __shared__ long long s_m[kDemapWin];
    __shared__ long long s_mbase;   // unwrap count of the window before the CTA's first
    __shared__ int s_red[NW];
    __shared__ int s_r;
    __shared__ unsigned s_cnt[C_NCNT];
    int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int w0 = blockIdx.x * kDemapWin;
    int wend = min(w0 + kDemapWin, g.nwin);
    if (tid < C_NCNT) s_cnt[tid] = 0;
    // Every load that does not depend on the unwrap counter is issued first: the
    // decisions of this warp's windows (symbols lane and lane + 32 of each), the
    // record of the warp's window `lane` (lanes < WPW) and the scan lane's phase
    // indices, so that their latencies overlap with each other and with the prefix.
    uint32_t dv[WPW];
#pragma unroll
    for (int i = 0; i < WPW; i++) {
        int wi = w0 + wid + NW * i;
        dv[i] = 0;
        if (wi < wend) {
            const uint8_t *d = dec + (long long)wi * kWin;
            dv[i] = (uint32_t)d[lane] | ((uint32_t)d[lane + 32] << 8);
        }
    }
    const int wr = w0 + wid + NW * lane;
    uint4 rc = make_uint4(0u, 0u, 0u, 0u);
    if (lane < WPW && wr < wend) rc = winrec[wr];
    if (QAM) {
        int have = dst->unwrap_have[uw_in];
        int blast = dst->unwrap_b[uw_in];
        long long mstart = have ? dst->unwrap_m[uw_in] : 0;
        const int ws = w0 + tid;   // the window scanned by thread tid < kDemapWin
        int sb = 0, sbp = 0;
        if (tid < kDemapWin && ws < wend) {
            sb = winb[ws];
            sbp = ws > 0 ? winb[ws - 1] : 0;
        }
        // prefix of increments over windows [0, w0): 16 windows per 16-byte load,
        // four loads in flight per thread
        const int nch = w0 / 16;
        int part = 0;
        for (int cb = tid; cb < nch; cb += 4 * kDemapThreads) {
            uint4 v[4];
            int pv[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                int c = cb + k * kDemapThreads;
                if (c < nch) {
                    v[k] = *reinterpret_cast<const uint4 *>(winb + 16 * c);
                    pv[k] = c ? winb[16 * c - 1] : 0;
                }
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                int c = cb + k * kDemapThreads;
                if (c >= nch) break;
                uint32_t wd[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
                int prev = c ? pv[k] : blast;
                bool use_first = (c > 0) || have;
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    int b = (wd[i >> 2] >> (8 * (i & 3))) & 0xFF;
                    if (i > 0 || use_first) part += unwrap_inc(prev, b, p.bps_b);
                    prev = b;
                }
            }
        }
        part = warp_sum_i(part);
        if (lane == 0) s_red[wid] = part;
        __syncthreads();
        long long pre = 0;
#pragma unroll
        for (int i = 0; i < NW; i++) pre += s_red[i];
        if (tid < 32) {   // inclusive scan of this CTA's increments
            int inc = 0;
            if (tid < kDemapWin && ws < wend && (ws > 0 || have)) inc = unwrap_inc(ws ? sbp : blast, sb, p.bps_b);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            if (tid < kDemapWin) s_m[tid] = mstart + pre + inc;
            if (tid == 0) s_mbase = mstart + pre;
        }
        if (resolve_amb) {
            // stream-start pi/2 ambiguity from the first amb_syms payload symbols:
            // the rotation r whose decoded symbols (rotation m_w + r) match the
            // transmitted ones best, ties to the lowest r; every CTA finds it alike
            if (tid < 32) {
                int nw = p.amb_syms / kWin;   // windows 0..nw-1 of this call (first payload call)
                int acc = 0;
                unsigned cnt[4] = {0, 0, 0, 0};
                for (int h = 0; h < 2; h++) {
                    int w = lane + 32 * h;
                    int v = (w < nw && w > 0) ? unwrap_inc(winb[w - 1], winb[w], p.bps_b) : 0;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        int t = __shfl_up_sync(0xffffffffu, v, o);
                        if (lane >= o) v += t;
                    }
                    int m = acc + v;
                    acc += __shfl_sync(0xffffffffu, v, 31);
                    if (w < nw) {
                        uint4 rw = winrec[w];
#pragma unroll
                        for (int r = 0; r < 4; r++) cnt[r] += rec_serr(rw, (m + r) & 3);
                    }
                }
                int best = 0;
                unsigned bc = 0;
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    unsigned c = warp_sum_i(cnt[r]);
                    if (r == 0 || c < bc) { bc = c; best = r; }
                }
                if (tid == 0) {
                    s_r = best;
                    if (blockIdx.x == 0) dst->amb_r = best;
                }
            }
        } else if (tid == 0) {
            s_r = dst->amb_r;
        }
    }
    __syncthreads();
    const int r = QAM ? s_r : 0;
    const long long amb_end = QAM ? (long long)p.ntrain + p.amb_syms : 0;
    // statistics: lane i < WPW selects from the record of the warp's window i
    if (lane < WPW && wr < wend) {
        long long k0 = g.pay_lo + (long long)wr * kWin;
        int qd = QAM ? (int)((s_m[wr - w0] + r) & 3) : 0;
        if (QAM && p.diff) {   // differential coding: errors are counted on the decoded bits below
            if (!(k0 < amb_end) && k0 + kWin <= g.score_end) atomicAdd(&s_cnt[C_NEAR], rc.w >> 8);
        } else if (!(QAM && k0 < amb_end) && k0 + kWin <= g.score_end) {
            int best = 0;
            unsigned be = rec_err(rc, qd);
#pragma unroll
            for (int rho = 1; rho < (QAM ? 4 : 1); rho++) {
                unsigned e = rec_err(rc, (qd + rho) & 3);
                if (e < be) { be = e; best = rho; }
            }
            int qb = (qd + best) & 3;
            atomicAdd(&s_cnt[C_BITERR], be);
            atomicAdd(&s_cnt[C_RAWERR], rec_err(rc, qd));
            atomicAdd(&s_cnt[C_SYMERR], rec_serr(rc, qb));
            atomicAdd(&s_cnt[C_SLIP], (unsigned)(best != 0));
            atomicAdd(&s_cnt[C_NEAR], rc.w >> 8);
            atomicAdd(&s_cnt[C_BITS], (unsigned)(BPS * kWin));
            atomicAdd(&s_cnt[C_SYMBOLS], (unsigned)kWin);
        }
        atomicAdd(&s_cnt[C_WINDOWS], 1u);
    }
    // output bits: Gray codes of the rotated decisions, byte b of a window holding
    // its bits [8b, 8b+8) MSB first, gathered from the owning lanes by shuffle.
    // Differential coding: the word of a symbol is the Gray code of its quadrant step
    // from the previous symbol, then (16QAM) its point's bits in the quadrant; the
    // previous symbol of a window's first one is the last of the window before it
    // (or the last of the previous call), and the decoded bits are scored here.
    const int sfirst = (8 * lane) / BPS, slast = (8 * lane + 7) / BPS;
    const int shift = BPS * (slast + 1) - (8 * lane + 8);
#pragma unroll
    for (int i = 0; i < WPW; i++) {
        int wi = w0 + wid + NW * i;
        if (wi >= wend) break;   // warp-uniform
        int qd = 0;
        if (QAM) {
            long long mw = s_m[wi - w0];
            qd = (int)((mw + r) & 3);
            if (dbg_win && lane == 0) dbg_win[wi].y = (float)mw;
        }
        uint32_t grp2 = 0;
        if (QAM && p.diff) {
            int qu[2], lb[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                int dvb = (dv[i] >> (8 * h)) & 0xFF;
                int LI = dvb & 7, LQ = (dvb >> 3) & 7;
                rot_t<MQ>(LI, LQ, qd);
                qu[h] = quad_t<MQ>(LI, LQ, lb[h]);
            }
            // quadrant of the symbol before this window's first
            int qprev0 = -1;
            if (lane == 0) {
                if (wi > 0) {
                    const long long mp = (wi - 1 >= w0) ? s_m[wi - 1 - w0] : s_mbase;
                    const int db = dec[(long long)(wi - 1) * kWin + kWin - 1];
                    int LI = db & 7, LQ = (db >> 3) & 7, lbx;
                    rot_t<MQ>(LI, LQ, (int)((mp + r) & 3));
                    qprev0 = quad_t<MQ>(LI, LQ, lbx);
                } else if (dst->diff_have[uw_in]) {
                    qprev0 = dst->diff_q[uw_in];
                }
            }
            const int up0 = __shfl_up_sync(0xffffffffu, qu[0], 1), up1 = __shfl_up_sync(0xffffffffu, qu[1], 1);
            const int last0 = __shfl_sync(0xffffffffu, qu[0], 31);
            int qp[2] = {lane ? up0 : (qprev0 < 0 ? qu[0] : qprev0), lane ? up1 : last0};
            const long long k0 = g.pay_lo + (long long)wi * kWin;
            const int pwin = (int)(((long long)BPS * k0) % 32767);
            unsigned ne = 0, se = 0;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int d = (qu[h] - qp[h]) & 3, gd = d ^ (d >> 1);
                const int w = (MQ == 4) ? ((gd << 2) | lb[h]) : gd;
                grp2 |= (uint32_t)w << (8 * h);
                const unsigned e = __popc((unsigned)(w ^ ref_bits<BPS>(prbs_bits, pwin + BPS * (lane + 32 * h))));
                ne += e;
                se += e > 0;
            }
            ne = warp_sum_i(ne);
            se = warp_sum_i(se);
            if (lane == 0 && !(k0 < amb_end) && k0 + kWin <= g.score_end) {
                atomicAdd(&s_cnt[C_BITERR], ne);
                atomicAdd(&s_cnt[C_RAWERR], ne);
                atomicAdd(&s_cnt[C_SYMERR], se);
                atomicAdd(&s_cnt[C_BITS], (unsigned)(BPS * kWin));
                atomicAdd(&s_cnt[C_SYMBOLS], (unsigned)kWin);
            }
            if (wi == g.nwin - 1 && lane == 31) {   // the next call's previous symbol
                dst->diff_q[uw_in ^ 1] = qu[1];
                dst->diff_have[uw_in ^ 1] = 1;
            }
        } else {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                int dvb = (dv[i] >> (8 * h)) & 0xFF;
                int LI = dvb & 7, LQ = QAM ? ((dvb >> 3) & 7) : 0;
                if (QAM) rot_t<MQ>(LI, LQ, qd);
                grp2 |= (uint32_t)(QAM ? ((gray(LI) << NB) | gray(LQ)) : gray(LI)) << (8 * h);
            }
        }
        uint32_t acc = 0;
#pragma unroll
        for (int j = 0; j < NS; j++) {
            int s = sfirst + j;
            uint32_t v = __shfl_sync(0xffffffffu, grp2, s & 31);
            if (s <= slast) acc = (acc << BPS) | (((s & 32) ? v >> 8 : v) & 0xFFu);
        }
        if (lane < NBYTES) bits_out[(long long)wi * NBYTES + lane] = (uint8_t)(acc >> shift);
    }
    __syncthreads();
    if (tid < C_NCNT && s_cnt[tid]) atomicAdd(&dst->cnt[tid], (unsigned long long)s_cnt[tid]);
    // carry the unwrap state to the next call
    if (QAM && wend == g.nwin && w0 < wend && tid == 0) {
        int o = uw_in ^ 1;
        dst->unwrap_have[o] = 1;
        dst->unwrap_b[o] = winb[g.nwin - 1];
        dst->unwrap_m[o] = s_m[g.nwin - 1 - w0];
    }
    if (g.lat && tid == 0) lat_end(g.lat, g.lat_slot);
}

cudaError_t launch_demap(const EqParams &p, const EqGeom &g, int resolve_amb, int uw_in, const uint8_t *dec,
                         const uint8_t *winb, const uint4 *winrec, float4 *dbg_win, uint8_t *bits_out,
                         const uint32_t *prbs_bits, DevState *dst, cudaStream_t st)
{
    unsigned grid = (unsigned)((g.nwin + kDemapWin - 1) / kDemapWin);
#define RX_DEMAP(Q, B, M)                                                                                   \
    k_demap<Q, B, M><<<grid, kDemapThreads, 0, st>>>(p, g, resolve_amb, uw_in, dec, winb, winrec, dbg_win,  \
                                                     bits_out, prbs_bits, dst)
    if (p.kk && p.mq == 4) RX_DEMAP(true, 4, 4);
    else if (p.kk) RX_DEMAP(true, 2, 2);
    else if (p.mq == 2) RX_DEMAP(false, 1, 2);
    else if (p.mq == 4) RX_DEMAP(false, 2, 4);
    else RX_DEMAP(false, 3, 8);
#undef RX_DEMAP
    return cudaGetLastError();
}

}  // namespace rxk
