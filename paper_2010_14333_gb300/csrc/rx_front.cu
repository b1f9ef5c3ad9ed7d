// Front end of the receiver: 12-bit unpack, Kramers-Kronig field reconstruction
// by overlap-save FFT Hilbert transform with carrier / gain reduction, and the
// matched filters (KK with downshift and 4 -> 2 decimation; PAM with DC removal).
//
// Paper: Sec. 2 -- 12-bit samples in 2^22-sample buffers; the KK front end takes
// the square root and logarithm inside the overlap-save step, recovers the phase
// with an FD Hilbert transform (FFT, IFFT), mixes it with the square-root term and
// downshifts (Fig. 1d: one thread per sample, amplitude and phase in, complex out);
// the signal is then filtered and reduced to 2 samples/symbol.
//
// Hilbert FFT layout.  One complex FFT of length N = 16 * N2 transforms two real
// overlap-save blocks at once (z = u_a + j u_b; the Hilbert multiplier -j sgn(k)
// is complex-linear, so phi_a + j phi_b = IFFT(h * FFT(z))).  N is split four-step
// style into a radix-16 pass over the stride-N2 index (K1a, registers only), an
// N2-point FFT per row with the multiplier and the inverse in shared memory (K1b),
// and the inverse radix-16 pass fused with sqrt/exp/field assembly (K1c).
#include <cooperative_groups.h>

#include "rx_common.cuh"
#include "rx_internal.cuh"

namespace rxk {

// ================================================================== unpack
// Two 12-bit samples per three bytes.  Eight samples (12 bytes, three aligned
// 32-bit words) per thread; the output is [history | this buffer] as uint16 codes.
__device__ __forceinline__ void decode_pair(uint32_t b0, uint32_t b1, uint32_t b2, int order,
                                            uint32_t &s0, uint32_t &s1)
{
    if (order == 0) {
        s0 = b0 | ((b1 & 0xFu) << 8);
        s1 = (b1 >> 4) | (b2 << 4);
    } else {
        s0 = (b0 << 4) | (b1 >> 4);
        s1 = ((b1 & 0xFu) << 8) | b2;
    }
}

__global__ void k_unpack(const uint8_t *__restrict__ in, uint16_t *__restrict__ codes,
                         const uint16_t *__restrict__ codes_prev, long long nb, int nhist,
                         long long prev_off, int first_call, int order, long long *s1,
                         long long *s2, LatRecord *lat, int lat_slot)
{
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (lat && g == 0) lat_start(lat, lat_slot);
    long long ngroups = nb / 8;
    long long lsum = 0, lsq = 0;
    if (g < ngroups) {
        const uint32_t *w = reinterpret_cast<const uint32_t *>(in + 12 * g);
        uint32_t w0 = __ldg(w), w1 = __ldg(w + 1), w2 = __ldg(w + 2);
        uint32_t by[12];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            by[i] = (w0 >> (8 * i)) & 0xFFu;
            by[4 + i] = (w1 >> (8 * i)) & 0xFFu;
            by[8 + i] = (w2 >> (8 * i)) & 0xFFu;
        }
        uint32_t s[8];
#pragma unroll
        for (int p = 0; p < 4; p++) decode_pair(by[3 * p], by[3 * p + 1], by[3 * p + 2], order, s[2 * p], s[2 * p + 1]);
        uint4 o;
        o.x = s[0] | (s[1] << 16);
        o.y = s[2] | (s[3] << 16);
        o.z = s[4] | (s[5] << 16);
        o.w = s[6] | (s[7] << 16);
        *reinterpret_cast<uint4 *>(codes + nhist + 8 * g) = o;
        if (s1) {
#pragma unroll
            for (int i = 0; i < 8; i++) { lsum += s[i]; lsq += (long long)s[i] * s[i]; }
        }
    } else if (g < ngroups + nhist) {
        long long j = g - ngroups;   // history sample j
        uint16_t v;
        if (first_call) {            // before the stream: first sample replicated
            uint32_t a, b;
            decode_pair(in[0], in[1], in[2], order, a, b);
            v = (uint16_t)a;
        } else {
            v = codes_prev[prev_off + j];
        }
        codes[j] = v;
    }
    if (s1) {
        // block reduction then one atomic per CTA (integer: exact and order free)
        __shared__ long long r1[32], r2[32];
        for (int o = 16; o; o >>= 1) {
            lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
            lsq += __shfl_xor_sync(0xffffffffu, lsq, o);
        }
        int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) { r1[wid] = lsum; r2[wid] = lsq; }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long a = 0, b = 0;
            for (int i = 0; i < (int)(blockDim.x >> 5); i++) { a += r1[i]; b += r2[i]; }
            if (a) atomicAdd(reinterpret_cast<unsigned long long *>(s1), (unsigned long long)a);
            if (b) atomicAdd(reinterpret_cast<unsigned long long *>(s2), (unsigned long long)b);
        }
    }
}

cudaError_t launch_unpack(const uint8_t *in, uint16_t *codes, const uint16_t *codes_prev,
                          long long nb, int nhist, long long prev_off, int first_call,
                          int pack_order, long long *s1, long long *s2, cudaStream_t st, LatRecord *lat,
                          int lat_slot)
{
    long long items = nb / 8 + nhist;
    int tpb = 256;
    unsigned grid = (unsigned)((items + tpb - 1) / tpb);
    k_unpack<<<grid, tpb, 0, st>>>(in, codes, codes_prev, nb, nhist, prev_off, first_call,
                                   pack_order, s1, s2, lat, lat_slot);
    return cudaGetLastError();
}

// ============================================================= KK Hilbert
// window start of overlap-save block j (the last block ends at the newest sample)
__device__ __forceinline__ long long ols_ws(const KkGeom &g, int j)
{
    return (j < g.J - 1) ? g.e_prev - g.V / 2 + (long long)j * g.hop : g.avail - g.N;
}
// kept positions [t_lo, t_hi) of block j inside its window
__device__ __forceinline__ void ols_kept(const KkGeom &g, int j, int &t_lo, int &t_hi)
{
    if (j < g.J - 1) {
        t_lo = g.V / 2;
        t_hi = g.V / 2 + g.hop;
    } else {
        int cnt = (int)(g.e_k - (g.e_prev + (long long)(g.J - 1) * g.hop));
        t_hi = g.N - g.V / 2;
        t_lo = t_hi - cnt;
    }
}

// u = ln(I)/2 - ln(2048)/2 (the constant is annihilated by the Hilbert transform
// and only keeps the FP32 FFT well scaled) and sqrt(I), I = code (0.5 for code 0):
// the codes are 12-bit, so both are exact lookup tables computed in double.
static int tw_split(int M)
{
    int m = 0;
    while ((1 << m) < M) m++;
    return (m + 1) / 2;
}
int kk_tw_entries(int M) { return (1 << tw_split(M)) + M / (1 << tw_split(M)); }

static void factored_twiddles(int M, float2 *out)
{
    const double pi = 3.14159265358979323846;
    int s = tw_split(M), lo = 1 << s, hi = M / lo;
    for (int a = 0; a < lo; a++) {
        double t = -2.0 * pi * (double)a / (double)M;
        out[a] = make_float2((float)cos(t), (float)sin(t));
    }
    for (int a = 0; a < hi; a++) {
        double t = -2.0 * pi * (double)a * (double)lo / (double)M;
        out[lo + a] = make_float2((float)cos(t), (float)sin(t));
    }
}

void kk_host_tables(int N, float *lnt, float2 *twN, float2 *twN2)
{
    for (int c = 0; c < kLutCodes; c++) {
        double I = c ? (double)c : 0.5;
        lnt[c] = (float)(0.5 * log(I / 2048.0));
    }
    factored_twiddles(N, twN);
    factored_twiddles(N / 16, twN2);
}

// factored twiddle table staged in shared memory
struct TwSmem {
    const float2 *lo, *hi;
    int s, mask;
    __device__ __forceinline__ float2 operator()(int a) const { return cmul(hi[a >> s], lo[a & mask]); }
};
// x[r] times W^(a r), r = 1..15 (conjugated twiddles when CONJ), W the table's root.
// Four twiddles come from the table (exponents a, 4a, 8a, 12a); the others are the
// powers w^2 = w w, w^3 = w^2 w of the first and the products W^(4qa) w^b, a few
// roundings more than a table value each.  The caller keeps 15 a below the table's
// length.
template <bool CONJ>
__device__ __forceinline__ void twiddle16(float2 (&x)[16], const TwSmem &tw, int a)
{
    const float2 w1 = tw(a), w2 = cmul(w1, w1), w3 = cmul(w2, w1);
    const float2 wb[4] = {make_float2(1.f, 0.f), w1, w2, w3};
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const float2 wq = q ? tw(4 * q * a) : make_float2(1.f, 0.f);
#pragma unroll
        for (int b = (q ? 0 : 1); b < 4; b++) {
            const float2 w = q ? (b ? cmul(wq, wb[b]) : wq) : wb[b];
            x[4 * q + b] = CONJ ? cmulc(x[4 * q + b], w) : cmul(x[4 * q + b], w);
        }
    }
}
__device__ __forceinline__ TwSmem stage_tw(const float2 *__restrict__ gtab, int M, float2 *sm)
{
    int m = 31 - __clz(M);
    int s = (m + 1) / 2, lo = 1 << s, n = lo + (M >> s);
    for (int i = threadIdx.x; i < n; i += blockDim.x) sm[i] = __ldg(gtab + i);
    TwSmem t;
    t.lo = sm;
    t.hi = sm + lo;
    t.s = s;
    t.mask = lo - 1;
    return t;
}

// Packed 12-bit input of the KK front end, read directly (the unpack is fused):
// stream sample n lives at byte 1.5 (n - cbase) of the virtual buffer
// [history (the nhist samples before this buffer) | this buffer].  A CTA covers
// 256 columns of a block pair; its 32 rows (2 blocks x 16 radix-16 rows) are 256
// consecutive samples each, whose 384 bytes start on a 48-byte boundary and are
// staged into shared memory with 16-byte loads.
struct KkPacked {
    const uint8_t *hist;   // packed history (nhist samples)
    const uint8_t *in;     // this buffer
    uint8_t *hist_next;    // history of the next call, or null
    long long hist_bytes;  // nhist * 3 / 2
    long long in_bytes;    // buf_len * 3 / 2
    int order, first_call;
    LatRecord *lat;        // latency record whose slot the call's first kernel stamps, or null
    int lat_slot;
};
constexpr int kRawWords = 100;   // 384 bytes of a row + spare word, 16-byte multiple

// (CTAs of kCtaK1 threads; the loop is unrolled so that every load issues before the
// first one is used)
template <int N2T>
__device__ __forceinline__ void stage_rows(const KkGeom &g, const KkPacked &pk, int pair, int c0,
                                           uint32_t (*raw)[kRawWords], bool hb)
{
    static_assert((32 * 24) % kCtaK1 == 0, "whole iterations");
#pragma unroll
    for (int i = threadIdx.x; i < 32 * 24; i += kCtaK1) {
        int row = i / 24, ch = i - 24 * (i / 24), blk = row >> 4, q = row & 15;
        if (blk && !hb) continue;
        long long n = ols_ws(g, 2 * pair + blk) + c0 + (long long)N2T * q;
        long long vb = (n - g.cbase) * 3 / 2 + 16 * ch;   // >= 0 for every window of the call
        const uint8_t *src = vb < pk.hist_bytes ? pk.hist + vb : pk.in + (vb - pk.hist_bytes);
        *reinterpret_cast<uint4 *>(&raw[row][4 * ch]) = __ldg(reinterpret_cast<const uint4 *>(src));
    }
}

// 12-bit code of column t of a staged row.  The row is a stream of 12-bit fields,
// two per three bytes.  In pack order 0 sample t fills bits [12 t, 12 t + 12) of the
// little-endian stream: one funnel shift of the two words that hold them and a mask.
// In pack order 1 the code's high nibble comes first: the two bytes that hold it are
// swapped, then a shift takes the high 12 bits (even t) or the low 12 bits (odd t).
// The word index and the shifts depend on t only, so a thread computes them once.
struct ColPos {
    int w;         // first of the two words
    unsigned fs;   // funnel shift
    unsigned ps;   // pack order 1: shift after the byte swap
};
template <int ORD>
__device__ __forceinline__ ColPos col_pos(int t)
{
    const int b = (3 * t) >> 1;   // first byte of the sample
    ColPos c;
    c.w = b >> 2;
    c.fs = 8 * (b & 3) + (ORD == 0 ? 4 * (t & 1) : 0);
    c.ps = ORD == 0 ? 0u : 4u * (1 - (t & 1));
    return c;
}
template <int ORD>
__device__ __forceinline__ uint32_t col_code(const uint32_t *rw, const ColPos &c)
{
    uint32_t v = __funnelshift_r(rw[c.w], rw[c.w + 1], c.fs);
    if (ORD == 1) v = __byte_perm(v, 0u, 0x4401) >> c.ps;   // (byte 0 << 8) | byte 1
    return v & 0xFFFu;
}

__device__ __forceinline__ uint32_t first_code(const KkPacked &pk, const DevState *dst)
{
    if (!pk.first_call) return (uint32_t)dst->first_code;
    uint32_t a, b;
    decode_pair(pk.in[0], pk.in[1], pk.in[2], pk.order, a, b);
    return a;
}

// K1a: unpack, u = ln(I)/2 by table, radix-16 pass over the stride-N2 index of two
// packed blocks, twiddle.  CTAs with blockIdx.y == npairs copy the next history.
// ORD: the pack order of the 12-bit input; N2T: the row length N / 16 (256 or 4096), so
// that the stride-N2 accesses take compile-time offsets.
template <int ORD, int N2T>
__global__ void __launch_bounds__(kCtaK1) k_kk_fwd(KkGeom g, KkPacked pk, float2 *__restrict__ fftws,
                                                  const KkTables tb, DevState *dst)
{
    __shared__ float2 s_tw[512];
    __shared__ __align__(16) uint32_t raw[32][kRawWords];
    __shared__ __align__(16) float s_ln[kLutCodes];
    int pair = blockIdx.y;
    if (pk.lat && blockIdx.x == 0 && pair == 0 && threadIdx.x == 0) lat_start(pk.lat, pk.lat_slot);
    if (pair == g.npairs) {
        // history of the next call: samples [avail - nhist, avail) = virtual bytes
        // [in_bytes, in_bytes + hist_bytes)
        long long nch = pk.hist_bytes / 16;
        for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nch; c += (long long)gridDim.x * blockDim.x) {
            long long vb = pk.in_bytes + 16 * c;
            const uint8_t *src = vb < pk.hist_bytes ? pk.hist + vb : pk.in + (vb - pk.hist_bytes);
            reinterpret_cast<uint4 *>(pk.hist_next)[c] = __ldg(reinterpret_cast<const uint4 *>(src));
        }
        return;
    }
    const TwSmem tw = stage_tw(tb.twN, g.N, s_tw);
    // the ln table in shared memory: a gather over 32 random codes costs a few bank
    // conflicts there instead of one L1 wavefront per distinct cache line
    for (int i = threadIdx.x; i < kLutCodes / 4; i += blockDim.x)
        reinterpret_cast<float4 *>(s_ln)[i] = __ldg(reinterpret_cast<const float4 *>(tb.lnt) + i);
    const int c0 = blockIdx.x * blockDim.x;
    const int jb = 2 * pair + 1;
    const bool hb = jb < g.J;
    stage_rows<N2T>(g, pk, pair, c0, raw, hb);
    const uint32_t c_first = first_code(pk, dst);
    if (pk.first_call && blockIdx.x == 0 && pair == 0 && threadIdx.x == 0) dst->first_code = (int)c_first;
    __syncthreads();
    const int t = threadIdx.x, n1 = c0 + t;
    const long long wa = ols_ws(g, 2 * pair) + c0 + t, wb = hb ? ols_ws(g, jb) + c0 + t : 0;
    // rows q below qa (qb) hold stream indices before the stream: the first code
    const int qa = wa < 0 ? (int)min((-wa + N2T - 1) / N2T, 16LL) : 0;
    const int qb = wb < 0 ? (int)min((-wb + N2T - 1) / N2T, 16LL) : 0;
    const ColPos cp = col_pos<ORD>(t);
    float2 x[16];
#pragma unroll
    for (int q = 0; q < 16; q++) {
        uint32_t ca = q < qa ? c_first : col_code<ORD>(raw[q], cp);
        float ua = s_ln[ca], ub = 0.f;
        if (hb) {
            uint32_t cb = q < qb ? c_first : col_code<ORD>(raw[16 + q], cp);
            ub = s_ln[cb];
        }
        x[q] = make_float2(ua, ub);
    }
    dft16<false>(x);
    twiddle16<false>(x, tw, n1);
    float2 *out = fftws + (size_t)pair * g.N + n1;
#pragma unroll
    for (int k2 = 0; k2 < 16; k2++) out[k2 * N2T] = x[k2];
}

// digit reversal of a P-digit base-16 index
template <int P>
__device__ __forceinline__ int drev16(int pos)
{
    int r = 0;
#pragma unroll
    for (int i = 0; i < P; i++) { r = (r << 4) | (pos & 15); pos >>= 4; }
    return r;
}

// Hilbert multiplier of bin k of an N-point spectrum: -j (0<k<N/2), +j (k>N/2), 0 at 0 and N/2
__device__ __forceinline__ float2 hilbert_mul(float2 v, int k, int N)
{
    if (k == 0 || 2 * k == N) return make_float2(0.f, 0.f);
    return (2 * k < N) ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
}

// K1b: per row k2 of a block pair, N2-point FFT (radix-16 decimation in
// frequency, digit-reversed output), Hilbert multiplier on the bins k = k2 + 16 k1,
// inverse FFT (radix-16 decimation in time back to natural order).  In place.
template <int P>
__global__ void __launch_bounds__(256, 3) k_kk_rows(KkGeom g, float2 *__restrict__ fftws,
                                                   const float2 *__restrict__ twN2g)
{
    constexpr int N2 = 1 << (4 * P);
    constexpr int TPR = N2 / 16;                  // threads per row
    constexpr int RPC = 256 / TPR;                // rows per CTA
    constexpr int SROW = N2 + N2 / 16;            // padded row in shared memory
    extern __shared__ float2 sm[];
    __shared__ float2 s_tw[128];
    const TwSmem tw2 = stage_tw(twN2g, N2, s_tw);
    __syncthreads();
    int lr = threadIdx.x / TPR, t = threadIdx.x % TPR;
    int row = blockIdx.x * RPC + lr;
    bool active = row < g.npairs * 16;
    int k2 = row & 15;
    float2 *s = sm + lr * SROW;
    float2 *d = fftws + (size_t)(active ? row : 0) * N2;
    float2 x[16];
    // forward pass 0 (sub-transform size N2) straight from global memory
#pragma unroll
    for (int r = 0; r < 16; r++) x[r] = active ? d[t + r * TPR] : make_float2(0.f, 0.f);
    dft16<false>(x);
    twiddle16<false>(x, tw2, t);
    if (P == 1) {
#pragma unroll
        for (int r = 0; r < 16; r++) x[r] = hilbert_mul(x[r], k2 + 16 * drev16<P>(r), g.N);
        dft16<true>(x);
        if (active)
#pragma unroll
            for (int r = 0; r < 16; r++) d[r] = x[r];
        return;
    }
    // a pass's 16 elements base + r stride sit at pad16(base) + r (stride + stride / 16)
    // when stride is a multiple of 16, or base is one and stride is 1: one pointer per
    // pass and compile-time offsets
    float2 *const s0 = s + pad16(t);
    constexpr int STR0 = TPR + TPR / 16;
#pragma unroll
    for (int r = 0; r < 16; r++) s0[r * STR0] = x[r];
    __syncthreads();
    // remaining forward passes; the last one is fused with the multiplier and the
    // first inverse pass
#pragma unroll
    for (int p = 1; p < P; p++) {
        const int M = N2 >> (4 * p), sub = M / 16, str = sub + sub / 16;
        int o = (t / sub) * M, j = t % sub;
        float2 *const sb = s + pad16(o + j);
#pragma unroll
        for (int r = 0; r < 16; r++) x[r] = sb[r * str];
        dft16<false>(x);
        if (p < P - 1) {
            twiddle16<false>(x, tw2, j * (N2 / M));
#pragma unroll
            for (int r = 0; r < 16; r++) sb[r * str] = x[r];
            __syncthreads();
        } else {
            // M = 16: positions o + r hold X[k2 + 16 * drev(o + r)]
#pragma unroll
            for (int r = 0; r < 16; r++) x[r] = hilbert_mul(x[r], k2 + 16 * drev16<P>(o + r), g.N);
            dft16<true>(x);
#pragma unroll
            for (int r = 0; r < 16; r++) sb[r] = x[r];   // sub = 1, j = 0
            __syncthreads();
        }
    }
    // inverse passes P-2 .. 1
#pragma unroll
    for (int p = P - 2; p >= 1; p--) {
        const int M = N2 >> (4 * p), sub = M / 16, str = sub + sub / 16;
        int o = (t / sub) * M, j = t % sub;
        float2 *const sb = s + pad16(o + j);
#pragma unroll
        for (int r = 0; r < 16; r++) x[r] = sb[r * str];
        twiddle16<true>(x, tw2, j * (N2 / M));
        dft16<true>(x);
#pragma unroll
        for (int r = 0; r < 16; r++) sb[r * str] = x[r];
        __syncthreads();
    }
    // inverse pass 0 to global memory
#pragma unroll
    for (int r = 0; r < 16; r++) x[r] = s0[r * STR0];
    twiddle16<true>(x, tw2, t);
    dft16<true>(x);
    if (active)
#pragma unroll
        for (int r = 0; r < 16; r++) d[t + r * TPR] = x[r];
}

// Carrier and intensity sums of a call, from which its carrier and gain follow.
// Each warp's FP32 sums of E become exact integers in units of 2^-24 (a warp's sum
// is below 2^17 in magnitude and a call holds at most 2^30 samples of |E| <= 64, so
// every total fits a signed 64-bit integer).  One 64-bit atomic per CTA and quantity
// adds them to the slot's totals.  Integer addition does not depend on order, so the
// totals, and the carrier, are the same whatever order the CTAs run in.  The CTA that
// takes the last ticket forms, in FP64, the carrier c = sum E / n, the mean intensity
// sum 2I / 2n and the gain 1 / sqrt(sps (mean I - |c|^2)), then clears the totals and
// the ticket for the slot's next call.
constexpr double kCarrierUnit = 16777216.0;   // 2^24
__device__ __forceinline__ void carrier_sums(const KkGeom &g, DevState *dst, float sre, float sim, int si2,
                                             int ncta)
{
    __shared__ long long s_q[3][32];
    sre = warp_sum_f(sre);
    sim = warp_sum_f(sim);
    si2 = warp_sum_i(si2);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_q[0][wid] = __double2ll_rn((double)sre * kCarrierUnit);
        s_q[1][wid] = __double2ll_rn((double)sim * kCarrierUnit);
        s_q[2][wid] = si2;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    long long a = 0, b = 0, c = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
        a += s_q[0][i];
        b += s_q[1][i];
        c += s_q[2][i];
    }
    unsigned long long *S = dst->csum[g.slot];
    atomicAdd(S + 0, (unsigned long long)a);
    atomicAdd(S + 1, (unsigned long long)b);
    atomicAdd(S + 2, (unsigned long long)c);
    __threadfence();
    if (atomicAdd(&dst->ticket[g.slot], 1u) != (unsigned)(ncta - 1)) return;
    __threadfence();
    const long long ta = (long long)atomicExch(S + 0, 0ull), tb = (long long)atomicExch(S + 1, 0ull),
                    tc = (long long)atomicExch(S + 2, 0ull);
    const double cnt = (double)(g.e_k - g.e_prev);
    const double cr = (double)ta / kCarrierUnit / cnt, ci = (double)tb / kCarrierUnit / cnt;
    const double ibar = (double)tc / (2.0 * cnt);
    const double P = ibar - (cr * cr + ci * ci);
    dst->cg[g.slot][0] = cr;
    dst->cg[g.slot][1] = ci;
    dst->cg[g.slot][2] = (P > 0.0) ? 1.0 / sqrt((double)g.sps * P) : 1.0;
    dst->ticket[g.slot] = 0u;
}

// K1c: inverse radix-16 pass, then for every kept output
// E = sqrt(I) * exp(j phi) (Fig. 1d), written at its stream position, and the
// per-call carrier / intensity sums (exact integer totals, carrier_sums).  The
// codes for sqrt(I) come from the same staged rows.  ORD: the pack order; N2T: the
// row length N / 16.
template <int ORD, int N2T>
__global__ void __launch_bounds__(kCtaK1) k_kk_inv(KkGeom g, KkPacked pk, const float2 *__restrict__ fftws,
                                                  const KkTables tb, float2 *__restrict__ E,
                                                  const float2 *__restrict__ E_prev, DevState *dst)
{
    __shared__ float2 s_tw[512];
    __shared__ __align__(16) uint32_t raw[32][kRawWords];
    const TwSmem tw = stage_tw(tb.twN, g.N, s_tw);
    int pair = blockIdx.y;
    const int c0 = blockIdx.x * blockDim.x;
    const bool hb = 2 * pair + 1 < g.J;
    stage_rows<N2T>(g, pk, pair, c0, raw, hb);
    const uint32_t c_first = first_code(pk, dst);
    float sre = 0.f, sim = 0.f;
    int si2 = 0;
    if (blockIdx.x == 0 && blockIdx.y == 0) {
        // field history for the matched filter: E[n], n in [e_prev - kEHist, e_prev)
        for (int i = threadIdx.x; i < kEHist; i += blockDim.x) {
            long long n = g.e_prev - kEHist + i;
            E[i] = (n < 0) ? make_float2(0.f, 0.f) : E_prev[n - g.ebase_prev];
        }
    }
    const int t = threadIdx.x, n1 = c0 + t;
    const ColPos cp = col_pos<ORD>(t);
    float2 x[16];
    const float2 *in = fftws + (size_t)pair * g.N + n1;
#pragma unroll
    for (int k2 = 0; k2 < 16; k2++) x[k2] = in[k2 * N2T];
    __syncthreads();   // staged twiddles and rows
    twiddle16<true>(x, tw, n1);
    dft16<true>(x);
    const float invN = 1.0f / (float)g.N;
#pragma unroll
    for (int half = 0; half < 2; half++) {
        int j = 2 * pair + half;
        if (j >= g.J) break;
        long long ws = ols_ws(g, j);
        int tlo, thi;
        ols_kept(g, j, tlo, thi);
        // 32-bit offsets from the block's first stream index: E row base, and the
        // local index below which the stream index is negative (before the stream)
        float2 *Eb = E + (ws - g.ebase);
        const int tneg = ws < 0 ? (int)(-ws) : 0;
#pragma unroll
        for (int q = 0; q < 16; q++) {
            int tt = n1 + N2T * q;
            if (tt < tlo || tt >= thi) continue;
            uint32_t code = tt < tneg ? c_first : col_code<ORD>(raw[16 * half + q], cp);
            float phi = (half ? x[q].y : x[q].x) * invN;
            float sn, cs;
            __sincosf(phi, &sn, &cs);   // |phi| < pi: absolute error <= 2^-21.41
            // the hardware square-root approximation (sqrt.approx.f32) in place of the
            // correctly rounded sequence; the field is held to the FP64 reference
            // within 1e-5 relative RMS
            float A = sqrt_approx(code ? (float)code : 0.5f);
            float2 e = make_float2(A * cs, A * sn);
            Eb[tt] = e;
            sre += e.x;
            sim += e.y;
            si2 += code ? 2 * (int)code : 1;
        }
    }
    carrier_sums(g, dst, sre, sim, si2, gridDim.x * gridDim.y);
}

// ====================================================== KK front end, fused
// One thread-block cluster of kClC CTAs per block pair computes the whole
// Hilbert transform of the pair in distributed shared memory (the 2^16-point
// case, N2 = 4096): CTA c owns rows k2 = 2c, 2c+1 of the 16 x 4096 four-step
// layout, padded as in K1b.
//   A  columns:  CTA c takes columns n1 in [512 c, 512 c + 512): 12-bit codes
//      straight from the packed input, u = ln(I)/2, radix-16 DFT over the
//      stride-N2 index, twiddle, each result stored into the shared memory of
//      the CTA that owns its row;
//   B  rows:     forward 4096-point FFT, Hilbert multiplier, inverse FFT of the
//      CTA's two rows in its own shared memory (the passes of K1b);
//   C  columns:  the 16 values of each of its columns gathered back from the
//      owners, inverse radix-16 DFT, E = sqrt(I) exp(j phi) for the kept
//      outputs and the carrier sums (the reduction of K1c).
// Cluster barriers separate the phases, so the 512 KB of a pair never leave the
// chip; global traffic is the packed input and the field.
constexpr int kClC = 8;
constexpr int kClThreads = 256;
constexpr int kClN2 = 4096;
constexpr int kClRow = kClN2 + kClN2 / 16;   // padded row
constexpr int kClCols = kClN2 / kClC;        // columns per CTA
constexpr size_t kClSmem = (size_t)(2 * kClRow + 512 + 128) * sizeof(float2);

// 12-bit codes of 32 consecutive stream samples (one per lane) starting at
// virtual-buffer offset t0 (a multiple of 32, so its 48 bytes start on 16 bytes
// and lie wholly in the history or in this buffer): lanes 0..11 load one word
// each, every lane takes its two bytes from the owners by shuffle.
__device__ __forceinline__ uint32_t warp_codes(const KkPacked &pk, long long t0, int lane)
{
    long long vb = (3 * t0) >> 1;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(vb < pk.hist_bytes ? pk.hist + vb
                                                                                : pk.in + (vb - pk.hist_bytes));
    uint32_t w = lane < 12 ? __ldg(src + lane) : 0u;
    int b = (3 * lane) >> 1;
    uint32_t w0 = __shfl_sync(0xffffffffu, w, b >> 2);
    uint32_t w1 = __shfl_sync(0xffffffffu, w, min((b >> 2) + 1, 31));
    uint32_t v = __funnelshift_r(w0, w1, 8 * (b & 3));
    uint32_t lo = v & 0xFFu, hi = (v >> 8) & 0xFFu;
    if (pk.order == 0) return (lane & 1) ? ((lo >> 4) | (hi << 4)) : (lo | ((hi & 0xFu) << 8));
    return (lane & 1) ? (((lo & 0xFu) << 8) | hi) : ((lo << 4) | (hi >> 4));
}

__global__ void __cluster_dims__(kClC, 1, 1) __launch_bounds__(kClThreads, 3)
    k_kk_cluster(KkGeom g, KkPacked pk, const KkTables tb, float2 *__restrict__ E,
                 const float2 *__restrict__ E_prev, DevState *dst)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ float2 smc[];
    float2 *rows = smc;                         // [2][kClRow]
    const TwSmem tw = stage_tw(tb.twN, g.N, smc + 2 * kClRow);
    const TwSmem tw2 = stage_tw(tb.twN2, kClN2, smc + 2 * kClRow + 512);
    const int c = (int)cl.block_rank();
    const int pair = blockIdx.x / kClC;
    const int t = threadIdx.x;
    if (pk.lat && blockIdx.x == 0 && t == 0) lat_start(pk.lat, pk.lat_slot);
    const bool hb = 2 * pair + 1 < g.J;
    const uint32_t c_first = first_code(pk, dst);
    if (pk.first_call && blockIdx.x == 0 && t == 0) dst->first_code = (int)c_first;
    // history of the next call (packed bytes [in_bytes, in_bytes + hist_bytes) of
    // the virtual buffer), spread over the grid
    if (pk.hist_next) {
        long long nch = pk.hist_bytes / 16;
        for (long long ch = (long long)blockIdx.x * blockDim.x + t; ch < nch; ch += (long long)gridDim.x * blockDim.x) {
            long long vb = pk.in_bytes + 16 * ch;
            const uint8_t *src = vb < pk.hist_bytes ? pk.hist + vb : pk.in + (vb - pk.hist_bytes);
            reinterpret_cast<uint4 *>(pk.hist_next)[ch] = __ldg(reinterpret_cast<const uint4 *>(src));
        }
    }
    if (blockIdx.x == 0)   // field history for the matched filter
        for (int i = t; i < kEHist; i += blockDim.x) {
            long long n = g.e_prev - kEHist + i;
            E[i] = (n < 0) ? make_float2(0.f, 0.f) : E_prev[n - g.ebase_prev];
        }
    __syncthreads();   // staged twiddles

    // ---- A: forward column DFTs, scattered to the row owners
    const long long wsa = ols_ws(g, 2 * pair), wsb = hb ? ols_ws(g, 2 * pair + 1) : 0;
    cl.sync();         // every CTA of the cluster is running before remote stores
#pragma unroll 1
    for (int h = 0; h < kClCols / kClThreads; h++) {
        const int n1 = c * kClCols + h * kClThreads + t;
        float2 x[16];
        const int lane = t & 31;
        const int n1w = n1 - lane;                  // first column of the warp
#pragma unroll
        for (int q = 0; q < 16; q++) {
            long long na = wsa + n1w + (long long)kClN2 * q;   // warp-uniform, a multiple of 32
            uint32_t ca = na < 0 ? c_first : warp_codes(pk, na - g.cbase, lane);
            float ub = 0.f;
            if (hb) {
                long long nb2 = wsb + n1w + (long long)kClN2 * q;
                ub = __ldg(tb.lnt + (nb2 < 0 ? c_first : warp_codes(pk, nb2 - g.cbase, lane)));
            }
            x[q] = make_float2(__ldg(tb.lnt + ca), ub);
        }
        dft16<false>(x);
#pragma unroll
        for (int k2 = 0; k2 < 16; k2++) {
            float2 *dstp = cl.map_shared_rank(rows + (k2 & 1) * kClRow, k2 >> 1);
            dstp[pad16(n1)] = k2 ? cmul(x[k2], tw(n1 * k2)) : x[0];
        }
    }
    cl.sync();

    // ---- B: the CTA's two rows, FFT / Hilbert / inverse FFT (passes of K1b, P = 3)
#pragma unroll 1
    for (int lr = 0; lr < 2; lr++) {
        const int k2 = 2 * c + lr;
        float2 *s = rows + lr * kClRow;
        float2 x[16];
#pragma unroll
        for (int r = 0; r < 16; r++) x[r] = s[pad16(t + r * 256)];
        dft16<false>(x);
#pragma unroll
        for (int r = 1; r < 16; r++) x[r] = cmul(x[r], tw2(t * r));
#pragma unroll
        for (int r = 0; r < 16; r++) s[pad16(t + r * 256)] = x[r];
        __syncthreads();
        {   // pass 1 (M = 256)
            int o = (t / 16) * 256, j = t % 16;
#pragma unroll
            for (int r = 0; r < 16; r++) x[r] = s[pad16(o + j + r * 16)];
            dft16<false>(x);
#pragma unroll
            for (int r = 1; r < 16; r++) x[r] = cmul(x[r], tw2(j * r * 16));
#pragma unroll
            for (int r = 0; r < 16; r++) s[pad16(o + j + r * 16)] = x[r];
        }
        __syncthreads();
        {   // pass 2 (M = 16), Hilbert multiplier on X[k2 + 16 drev(o + r)], first inverse pass
            int o = t * 16;
#pragma unroll
            for (int r = 0; r < 16; r++) x[r] = s[pad16(o + r)];
            dft16<false>(x);
#pragma unroll
            for (int r = 0; r < 16; r++) x[r] = hilbert_mul(x[r], k2 + 16 * drev16<3>(o + r), g.N);
            dft16<true>(x);
#pragma unroll
            for (int r = 0; r < 16; r++) s[pad16(o + r)] = x[r];
        }
        __syncthreads();
        {   // inverse pass 1
            int o = (t / 16) * 256, j = t % 16;
#pragma unroll
            for (int r = 0; r < 16; r++) {
                x[r] = s[pad16(o + j + r * 16)];
                if (r) x[r] = cmulc(x[r], tw2(j * r * 16));
            }
            dft16<true>(x);
#pragma unroll
            for (int r = 0; r < 16; r++) s[pad16(o + j + r * 16)] = x[r];
        }
        __syncthreads();
        // inverse pass 0, in place
#pragma unroll
        for (int r = 0; r < 16; r++) {
            x[r] = s[pad16(t + r * 256)];
            if (r) x[r] = cmulc(x[r], tw2(t * r));
        }
        dft16<true>(x);
#pragma unroll
        for (int r = 0; r < 16; r++) s[pad16(t + r * 256)] = x[r];
    }
    cl.sync();

    // ---- C: inverse column DFTs from the row owners, field and carrier sums
    float sre = 0.f, sim = 0.f;
    int si2 = 0;
    const float invN = 1.0f / (float)g.N;
#pragma unroll 1
    for (int h = 0; h < kClCols / kClThreads; h++) {
        const int n1 = c * kClCols + h * kClThreads + t;
        float2 x[16];
#pragma unroll
        for (int k2 = 0; k2 < 16; k2++) {
            const float2 *srcp = cl.map_shared_rank(rows + (k2 & 1) * kClRow, k2 >> 1);
            x[k2] = srcp[pad16(n1)];
        }
#pragma unroll
        for (int k2 = 1; k2 < 16; k2++) x[k2] = cmulc(x[k2], tw(n1 * k2));
        dft16<true>(x);
#pragma unroll
        for (int half = 0; half < 2; half++) {
            int j = 2 * pair + half;
            if (j >= g.J) break;
            long long ws = half ? wsb : wsa;
            int tlo, thi;
            ols_kept(g, j, tlo, thi);
            const int lane = t & 31;
#pragma unroll
            for (int q = 0; q < 16; q++) {
                int tt = n1 + kClN2 * q;
                int tw0 = tt - lane;                    // warp-uniform
                if (tw0 + 31 < tlo || tw0 >= thi) continue;
                long long n = ws + tt;
                long long nw = ws + tw0;
                uint32_t code = nw < 0 ? c_first : warp_codes(pk, nw - g.cbase, lane);
                if (tt < tlo || tt >= thi) continue;
                float phi = (half ? x[q].y : x[q].x) * invN;
                float sn, cs;
                __sincosf(phi, &sn, &cs);   // |phi| < pi: absolute error <= 2^-21.41
                float A = sqrt_approx(code ? (float)code : 0.5f);
                float2 e = make_float2(A * cs, A * sn);
                E[n - g.ebase] = e;
                sre += e.x;
                sim += e.y;
                si2 += code ? 2 * (int)code : 1;
            }
        }
    }
    cl.sync();   // no CTA leaves while its rows may still be read

    carrier_sums(g, dst, sre, sim, si2, gridDim.x);
}

__global__ void k_kk_hist(KkPacked pk)
{
    if (pk.lat && blockIdx.x == 0 && threadIdx.x == 0) lat_start(pk.lat, pk.lat_slot);
    long long nch = pk.hist_bytes / 16;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nch; c += (long long)gridDim.x * blockDim.x) {
        long long vb = pk.in_bytes + 16 * c;
        const uint8_t *src = vb < pk.hist_bytes ? pk.hist + vb : pk.in + (vb - pk.hist_bytes);
        reinterpret_cast<uint4 *>(pk.hist_next)[c] = __ldg(reinterpret_cast<const uint4 *>(src));
    }
}

cudaError_t launch_kk_hist(const KkInput &inp, cudaStream_t st, const KkSync &sync)
{
    if (sync.wait_fwd) cudaStreamWaitEvent(st, sync.wait_fwd, 0);
    KkPacked pk;
    pk.hist = inp.hist;
    pk.in = inp.in;
    pk.hist_next = inp.hist_next;
    pk.hist_bytes = inp.hist_bytes;
    pk.in_bytes = inp.in_bytes;
    pk.order = inp.order;
    pk.first_call = inp.first_call;
    pk.lat = inp.lat;
    pk.lat_slot = inp.lat_slot;
    k_kk_hist<<<32, 256, 0, st>>>(pk);
    if (sync.rec_fwd) cudaEventRecord(sync.rec_fwd, st);
    return cudaGetLastError();
}

cudaError_t prepare_kk_front()
{
    return cudaFuncSetAttribute(k_kk_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClSmem);
}

cudaError_t launch_kk_front(const KkGeom &g, const KkInput &inp, float2 *fftws, const KkTables &tb,
                            float2 *E, const float2 *E_prev, DevState *dst, cudaStream_t st, void *prof,
                            const KkSync &sync)
{
    KkPacked pk;
    pk.hist = inp.hist;
    pk.in = inp.in;
    pk.hist_next = inp.hist_next;
    pk.hist_bytes = inp.hist_bytes;
    pk.in_bytes = inp.in_bytes;
    pk.order = inp.order;
    pk.first_call = inp.first_call;
    pk.lat = inp.lat;
    pk.lat_slot = inp.lat_slot;
    if (g.N2 == kClN2 && g.fused) {
        // 2^16-point blocks: the fused cluster kernel (profiled as the K1a stage)
        if (sync.wait_fwd) cudaStreamWaitEvent(st, sync.wait_fwd, 0);
        if (sync.wait_inv) cudaStreamWaitEvent(st, sync.wait_inv, 0);
        prof_stage(prof, 1, st);
        k_kk_cluster<<<g.npairs * kClC, kClThreads, kClSmem, st>>>(g, pk, tb, E, E_prev, dst);
        if (sync.rec_fwd) cudaEventRecord(sync.rec_fwd, st);
        prof_stage(prof, -2, st);
        prof_stage(prof, -3, st);
        prof_stage(prof, -4, st);
        return cudaGetLastError();
    }
    dim3 grid(g.N2 / kCtaK1, g.npairs);
    dim3 grid_a(g.N2 / kCtaK1, g.npairs + (inp.hist_next ? 1 : 0));
    if (sync.wait_fwd) cudaStreamWaitEvent(st, sync.wait_fwd, 0);
    prof_stage(prof, 1, st);
    if (g.N2 != 4096 && g.N2 != 256) return cudaErrorInvalidValue;   // N is 65536 or 4096
    const bool long_rows = g.N2 == 4096;
    if (pk.order) {
        if (long_rows) k_kk_fwd<1, 4096><<<grid_a, kCtaK1, 0, st>>>(g, pk, fftws, tb, dst);
        else k_kk_fwd<1, 256><<<grid_a, kCtaK1, 0, st>>>(g, pk, fftws, tb, dst);
    } else {
        if (long_rows) k_kk_fwd<0, 4096><<<grid_a, kCtaK1, 0, st>>>(g, pk, fftws, tb, dst);
        else k_kk_fwd<0, 256><<<grid_a, kCtaK1, 0, st>>>(g, pk, fftws, tb, dst);
    }
    if (sync.rec_fwd) cudaEventRecord(sync.rec_fwd, st);
    prof_stage(prof, -2, st);
    int rows = g.npairs * 16;
    if (g.N2 == 4096) {
        size_t smem = (size_t)(4096 + 256) * sizeof(float2);
        k_kk_rows<3><<<rows, 256, smem, st>>>(g, fftws, tb.twN2);
    } else if (g.N2 == 256) {
        size_t smem = (size_t)16 * (256 + 16) * sizeof(float2);
        k_kk_rows<2><<<(rows + 15) / 16, 256, smem, st>>>(g, fftws, tb.twN2);
    } else {
        k_kk_rows<1><<<(rows + 255) / 256, 256, 0, st>>>(g, fftws, tb.twN2);
    }
    if (sync.wait_inv) cudaStreamWaitEvent(st, sync.wait_inv, 0);
    prof_stage(prof, -3, st);
    if (pk.order) {
        if (long_rows) k_kk_inv<1, 4096><<<grid, kCtaK1, 0, st>>>(g, pk, fftws, tb, E, E_prev, dst);
        else k_kk_inv<1, 256><<<grid, kCtaK1, 0, st>>>(g, pk, fftws, tb, E, E_prev, dst);
    } else {
        if (long_rows) k_kk_inv<0, 4096><<<grid, kCtaK1, 0, st>>>(g, pk, fftws, tb, E, E_prev, dst);
        else k_kk_inv<0, 256><<<grid, kCtaK1, 0, st>>>(g, pk, fftws, tb, E, E_prev, dst);
    }
    prof_stage(prof, -4, st);
    return cudaGetLastError();
}

// ============================================================ KK matched filter
// y[m] = g * sum_i h_i * (E[2m - i] - c) * exp(-j 2 pi ds (2m - i)),  x[n < 0] = 0.
// 256 outputs per CTA from a shared-memory tile of the carrier-removed,
// downshifted field.  CTA 0 also carries the equaliser history [ybase, f_prev).
constexpr int kMfOut = 256;

__global__ void __launch_bounds__(kMfOut) k_kk_mf(const float2 *__restrict__ E, long long ebase, long long e_k,
                                                 long long f_prev, long long f_k, const float *__restrict__ rrc,
                                                 int hmf, const float2 *__restrict__ ds_tab, int ds_num,
                                                 int ds_den, const double *__restrict__ cg,
                                                 float2 *__restrict__ Y, long long ybase,
                                                 const float2 *__restrict__ Y_prev, long long ybase_prev)
{
    extern __shared__ float2 xs[];
    long long m0 = f_prev + (long long)blockIdx.x * kMfOut;
    int L = 2 * kMfOut + 2 * hmf;
    float2 c = make_float2((float)cg[0], (float)cg[1]);
    float gn = (float)cg[2];
    long long n0 = 2 * m0 - hmf;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        long long n = n0 + i;
        float2 v = make_float2(0.f, 0.f);
        if (n >= 0 && n < e_k) {
            int p = (int)(((n % ds_den) * ds_num) % ds_den);
            v = cmul(csub(E[n - ebase], c), __ldg(ds_tab + p));
        }
        xs[i] = v;
    }
    if (blockIdx.x == 0) {
        for (long long m = ybase + threadIdx.x; m < f_prev; m += blockDim.x)
            Y[m - ybase] = (m < 0) ? make_float2(0.f, 0.f) : Y_prev[m - ybase_prev];
    }
    __syncthreads();
    long long m = m0 + threadIdx.x;
    if (m >= f_k) return;
    const float2 *xc = xs + 2 * threadIdx.x + hmf;
    float ar = 0.f, ai = 0.f;
    for (int i = -hmf; i <= hmf; i++) {
        float h = __ldg(rrc + i + hmf);
        float2 v = xc[-i];
        ar = fmaf(h, v.x, ar);
        ai = fmaf(h, v.y, ai);
    }
    Y[m - ybase] = make_float2(gn * ar, gn * ai);
}

// Register-tiled form for a compile-time half length HMF (even).  With the tile
// starting at n0 = 2 m0 - HMF, the pairs P[p] = (x[n0 + 2p], x[n0 + 2p + 1])
// turn the decimating filter into two plain FIRs over the pair index:
//   y[m0 + j] = g * sum_{u=0..HMF} (ge[u] P[j+u].first + go[u] P[j+u].second)
// with ge[u] = h[HMF - 2u], go[u] = h[HMF - 2u - 1].  Each thread computes 8
// consecutive outputs from a sliding window of 8 pairs held in registers (one
// 16-byte shared load per tap); the pair layout keeps one spare slot per 8 pairs,
// which makes the stride-8-pair loads of a warp free of bank conflicts.  The real
// and imaginary parts of an output accumulate as one packed FP32 pair (one
// fma.rn.f32x2 per tap and output, the same roundings as two scalar FMAs in the
// same order); the taps sit in shared memory as (ge, ge, go, go).
template <int HMF>
struct MfTaps {
    float ge[HMF + 1];
    float go[HMF];
};

constexpr int kMfThreads = 128, kMfR = 8, kMfTileOut = kMfThreads * kMfR;
__host__ __device__ __forceinline__ int pad8(int p) { return p + (p >> 3); }

template <int HMF>
__global__ void __launch_bounds__(kMfThreads) k_kk_mf_t(const float2 *__restrict__ E, long long ebase,
                                                       long long e_k, long long f_prev, long long f_k,
                                                       const MfTaps<HMF> taps, const float2 *__restrict__ ds_tab,
                                                       int ds_num, int ds_den, const double *__restrict__ cg,
                                                       float2 *__restrict__ Y, long long ybase,
                                                       const float2 *__restrict__ Y_prev, long long ybase_prev)
{
    constexpr int NPAIR = kMfTileOut + HMF + kMfR;
    extern __shared__ float4 pr[];     // padded pair tile
    __shared__ float4 s_tp[HMF + 1];   // (ge, ge, go, go) per tap index u (go[HMF] = 0)
    long long m0 = f_prev + (long long)blockIdx.x * kMfTileOut;
    long long n0 = 2 * m0 - HMF;
    const float2 c = make_float2((float)cg[0], (float)cg[1]);
    const float gn = (float)cg[2];
    for (int u = threadIdx.x; u <= HMF; u += kMfThreads) {
        const float ho = u < HMF ? taps.go[u] : 0.f;
        s_tp[u] = make_float4(taps.ge[u], taps.ge[u], ho, ho);
    }
    // integer phase index of the downshift, advanced incrementally
    int idx = (int)((((n0 % ds_den) + ds_den) % ds_den + 2LL * threadIdx.x) % ds_den);
    idx = (int)(((long long)idx * ds_num) % ds_den);
    const int step = (int)((2LL * kMfThreads * ds_num) % ds_den), odd = ds_num % ds_den;
    // unrolled (a compile-time trip count): every iteration's loads can issue before
    // the first one is used
#pragma unroll
    for (int pp = threadIdx.x; pp < NPAIR; pp += kMfThreads) {
        long long n = n0 + 2 * pp;
        float2 a = make_float2(0.f, 0.f), b = a;
        if (n >= 0 && n < e_k) a = cmul(csub(E[n - ebase], c), __ldg(ds_tab + idx));
        int idx1 = idx + odd;
        idx1 = idx1 >= ds_den ? idx1 - ds_den : idx1;
        if (n + 1 >= 0 && n + 1 < e_k) b = cmul(csub(E[n + 1 - ebase], c), __ldg(ds_tab + idx1));
        pr[pad8(pp)] = make_float4(a.x, a.y, b.x, b.y);
        idx += step;
        idx = idx >= ds_den ? idx - ds_den : idx;
    }
    if (blockIdx.x == 0) {
        for (long long m = ybase + threadIdx.x; m < f_prev; m += blockDim.x)
            Y[m - ybase] = (m < 0) ? make_float2(0.f, 0.f) : Y_prev[m - ybase_prev];
    }
    __syncthreads();
    const ulonglong2 *prp = reinterpret_cast<const ulonglong2 *>(pr);
    const ulonglong2 *tpp = reinterpret_cast<const ulonglong2 *>(s_tp);
    const int j0 = kMfR * threadIdx.x;
    ulonglong2 win[kMfR];
#pragma unroll
    for (int r = 0; r < kMfR; r++) win[r] = prp[pad8(j0 + r)];
    f2x acc[kMfR];
#pragma unroll
    for (int r = 0; r < kMfR; r++) acc[r] = 0ull;   // (+0, +0)
#pragma unroll
    for (int u = 0; u <= HMF; u++) {
        const ulonglong2 T = tpp[u];
#pragma unroll
        for (int r = 0; r < kMfR; r++) acc[r] = f2_fma(T.x, win[r].x, acc[r]);
        if (u < HMF) {
#pragma unroll
            for (int r = 0; r < kMfR; r++) acc[r] = f2_fma(T.y, win[r].y, acc[r]);
#pragma unroll
            for (int r = 0; r < kMfR - 1; r++) win[r] = win[r + 1];
            win[kMfR - 1] = prp[pad8(j0 + u + kMfR)];
        }
    }
    const f2x g2 = f2_pack(gn, gn);
    float2 out[kMfR];
#pragma unroll
    for (int r = 0; r < kMfR; r++) out[r] = f2_unpack(f2_mul(g2, acc[r]));
    long long mb = m0 + j0;
    if (mb + kMfR <= f_k) {
        float4 *o = reinterpret_cast<float4 *>(Y + (mb - ybase));
        bool al = (((uintptr_t)o) & 15) == 0;
        if (al) {
#pragma unroll
            for (int r = 0; r < kMfR; r += 2)
                o[r / 2] = make_float4(out[r].x, out[r].y, out[r + 1].x, out[r + 1].y);
        } else {
#pragma unroll
            for (int r = 0; r < kMfR; r++) Y[mb + r - ybase] = out[r];
        }
    } else {
#pragma unroll
        for (int r = 0; r < kMfR; r++)
            if (mb + r < f_k) Y[mb + r - ybase] = out[r];
    }
}

cudaError_t launch_kk_mf(const float2 *E, long long ebase, long long e_k, long long f_prev,
                         long long f_k, const float *rrc, int hmf, const float2 *ds_tab,
                         int ds_num, int ds_den, const double *cg, float2 *Y, long long ybase,
                         const float2 *Y_prev, long long ybase_prev, cudaStream_t st,
                         const float *rrc_host)
{
    long long n = f_k - f_prev;
    if (hmf == 32 && rrc_host) {
        MfTaps<32> t;
        for (int u = 0; u <= 32; u++) t.ge[u] = rrc_host[32 + (32 - 2 * u)];
        for (int u = 0; u < 32; u++) t.go[u] = rrc_host[32 + (32 - 2 * u - 1)];
        unsigned grid = (unsigned)((n + kMfTileOut - 1) / kMfTileOut);
        size_t smem = (size_t)pad8(kMfTileOut + 32 + kMfR) * sizeof(float4) + 16;
        k_kk_mf_t<32><<<grid, kMfThreads, smem, st>>>(E, ebase, e_k, f_prev, f_k, t, ds_tab, ds_num, ds_den, cg,
                                                      Y, ybase, Y_prev, ybase_prev);
        return cudaGetLastError();
    }
    unsigned grid = (unsigned)((n + kMfOut - 1) / kMfOut);
    size_t smem = (size_t)(2 * kMfOut + 2 * hmf) * sizeof(float2);
    k_kk_mf<<<grid, kMfOut, smem, st>>>(E, ebase, e_k, f_prev, f_k, rrc, hmf, ds_tab, ds_num,
                                        ds_den, cg, Y, ybase, Y_prev, ybase_prev);
    return cudaGetLastError();
}

// ================================================ resampler to the transmitter's grid
// The ADC runs on its own clock (Sec. 2: the DSP recovers the clock phase).  Nominal
// sample m of the transmitter's grid lies at ADC position psi_m / 2^32 with the exact
// integer accumulator psi_m = psi_{m0} + (m - m0) step; its field is the 16-tap
// Hann-windowed sinc interpolation sum_{j=-7..8} c_j(mu) E[i + j] of the
// reconstructed field at i = floor(psi / 2^32) and the fraction mu rounded down to
// 10 bits (a 1024 x 16 table).  The host splits psi_{m0} (m0 = this call's first
// output) into its integer part i0 and fraction f0, so every offset inside a call
// fits in 64 bits.  One CTA per kRsOut outputs stages their ADC window in shared
// memory first.
constexpr int kRsThreads = 256, kRsPer = 4, kRsOut = kRsThreads * kRsPer, kRsWin = kRsOut + kRsOut / 64 + 24;

__global__ void __launch_bounds__(kRsThreads) k_kk_resample(const float2 *__restrict__ E, long long ebase,
                                                       long long r_prev, long long r_k, long long i0,
                                                       unsigned f0, long long step, const float *__restrict__ tab,
                                                       float2 *__restrict__ R, long long rbase,
                                                       const float2 *__restrict__ R_prev, long long rbase_prev)
{
    __shared__ float2 xs[kRsWin];
    const long long m0 = r_prev + (long long)blockIdx.x * kRsOut;
    // the CTA's first output in integer part and fraction; with step = 2^32 + delta
    // (|delta| < 2^32 / 64) thread t sits at i_b + t + floor((f_b + t delta) / 2^32)
    const long long accb = (long long)f0 + (m0 - r_prev) * step;
    const long long i_b = i0 + (accb >> 32);
    const long long f_b = accb & 0xFFFFFFFFLL;
    const int delta = (int)(step - (1LL << 32));
    const int nout = (int)min((long long)kRsOut, r_k - m0);
    const long long a0 = i_b - 7;
    const int len = (nout - 1) + (int)((f_b + (long long)(nout - 1) * delta) >> 32) + 16;
    for (int t = threadIdx.x; t < len && t < kRsWin; t += blockDim.x) {
        const long long n = a0 + t;
        xs[t] = n < 0 ? make_float2(0.f, 0.f) : E[n - ebase];
    }
    if (blockIdx.x == 0)   // the filter's history on the nominal grid
        for (long long m = rbase + threadIdx.x; m < r_prev; m += blockDim.x)
            R[m - rbase] = (m < 0) ? make_float2(0.f, 0.f) : R_prev[m - rbase_prev];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRsPer; k++) {   // outputs t, t + 256, ...: coalesced stores
        const int t = threadIdx.x + kRsThreads * k;
        if (t >= nout) return;
        const long long v = f_b + (long long)t * delta;   // |v| < 2^39
        const int li = t + (int)(v >> 32);                  // local index of E[i - 7]
        const float4 *c4 = reinterpret_cast<const float4 *>(tab + ((unsigned)(v & 0xFFFFFFFFLL) >> 22) * 16);
        float cj[16];
#pragma unroll
        for (int q = 0; q < 4; q++) {   // the 64-byte row in four 16-byte loads
            const float4 w = __ldg(c4 + q);
            cj[4 * q] = w.x;
            cj[4 * q + 1] = w.y;
            cj[4 * q + 2] = w.z;
            cj[4 * q + 3] = w.w;
        }
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const float2 x = xs[li + j];
            re = fmaf(cj[j], x.x, re);
            im = fmaf(cj[j], x.y, im);
        }
        R[m0 + t - rbase] = make_float2(re, im);
    }
}

cudaError_t launch_kk_resample(const float2 *E, long long ebase, long long r_prev, long long r_k, long long i0,
                               unsigned f0, long long step, const float *tab, float2 *R, long long rbase,
                               const float2 *R_prev, long long rbase_prev, cudaStream_t st)
{
    // the window of kRsOut outputs spans at most kRsOut step / 2^32 + 17 ADC samples
    if (step < (1LL << 32) - (1LL << 32) / 64 || step > (1LL << 32) + (1LL << 32) / 64) return cudaErrorInvalidValue;
    const long long n = r_k - r_prev;
    if (n <= 0) return cudaSuccess;
    k_kk_resample<<<(unsigned)((n + kRsOut - 1) / kRsOut), kRsThreads, 0, st>>>(E, ebase, r_prev, r_k, i0, f0, step, tab,
                                                                           R, rbase, R_prev, rbase_prev);
    return cudaGetLastError();
}

// ============================================ frequency-domain reduction (KK)
// The paper's form of the filter before the equaliser (Sec. 2, KK chain): a
// static filter applied in the frequency domain on overlap-save blocks of N =
// fd_n samples with hop N/2, and an N/2-point inverse transform of the kept bins
// -N/4 <= k < N/4 as the downsampler to 2 samples/symbol.  One CTA per block b:
//   - the N inputs from stream index N/2 b - N/4 (carrier removed, downshifted by
//     the exact integer phase; zero before the stream start) are staged in
//     shared memory;
//   - a radix-4 Stockham FFT (natural order in and out, two ping-pong buffers,
//     a last radix-2 pass when log2 N is odd) transforms them;
//   - the kept bins times the filter response (pre-scaled by 1/N) form the
//     N/2-point spectrum, which the inverse Stockham FFT brings back;
//   - the central half, N/4 outputs, leaves at 2 samples/symbol times the gain.
constexpr int kFdThreads = 128;

// Stockham passes of an n-point transform (n = N or N/2) on shared buffers a, b;
// tw is the N-point table e^{-2 pi i t / N}; returns the buffer with the result
template <bool INV>
__device__ float2 *stockham(float2 *a, float2 *b, int n, int N, const float2 *__restrict__ tw)
{
    int ns = 1;
    for (; ns * 4 <= n; ns *= 4) {
        const int q4 = n >> 2, ts = N / (4 * ns);
        for (int j = threadIdx.x; j < q4; j += blockDim.x) {
            const int k = j & (ns - 1);
            float2 v0 = a[j], v1 = a[j + q4], v2 = a[j + 2 * q4], v3 = a[j + 3 * q4];
            if (ns > 1) {
                float2 w1 = __ldg(tw + k * ts), w2 = __ldg(tw + 2 * k * ts), w3 = __ldg(tw + 3 * k * ts);
                if (INV) {
                    w1 = cconj(w1);
                    w2 = cconj(w2);
                    w3 = cconj(w3);
                }
                v1 = cmul(v1, w1);
                v2 = cmul(v2, w2);
                v3 = cmul(v3, w3);
            }
            dft4<INV>(v0, v1, v2, v3);
            const int o = ((j - k) << 2) + k;
            b[o] = v0;
            b[o + ns] = v1;
            b[o + 2 * ns] = v2;
            b[o + 3 * ns] = v3;
        }
        __syncthreads();
        float2 *t = a;
        a = b;
        b = t;
    }
    if (ns < n) {   // one radix-2 pass
        const int h2 = n >> 1, ts = N / (2 * ns);
        for (int j = threadIdx.x; j < h2; j += blockDim.x) {
            const int k = j & (ns - 1);
            float2 w = __ldg(tw + k * ts);
            if (INV) w = cconj(w);
            const float2 v0 = a[j], v1 = cmul(a[j + h2], w);
            const int o = ((j - k) << 1) + k;
            b[o] = cadd(v0, v1);
            b[o + ns] = csub(v0, v1);
        }
        __syncthreads();
        a = b;
    }
    return a;
}

__global__ void __launch_bounds__(kFdThreads) k_kk_fdmf(const float2 *__restrict__ E, long long ebase,
                                                       long long b_first, int N, const float2 *__restrict__ H,
                                                       const float2 *__restrict__ tw,
                                                       const float2 *__restrict__ ds_tab, int ds_num, int ds_den,
                                                       const double *__restrict__ cg, float2 *__restrict__ Y,
                                                       long long ybase, long long f_prev,
                                                       const float2 *__restrict__ Y_prev, long long ybase_prev,
                                                       float2 *__restrict__ clk, int wbin)
{
    extern __shared__ float2 fbuf[];   // [2][N]
    float2 *a = fbuf, *b = fbuf + N;
    const long long blk = b_first + blockIdx.x;
    const long long n0 = (N / 2) * blk - N / 4;   // stream index of the block's first input
    const float2 c = make_float2((float)cg[0], (float)cg[1]);
    const float gn = (float)cg[2];
    // integer phase index of the downshift: p(n) = n ds_num mod ds_den, advanced by the thread stride
    long long r0 = (n0 + threadIdx.x) % ds_den;
    if (r0 < 0) r0 += ds_den;
    int p = (int)((r0 * ds_num) % ds_den);
    const int step = (int)(((long long)kFdThreads * ds_num) % ds_den);
    for (int t = threadIdx.x; t < N; t += kFdThreads) {
        const long long n = n0 + t;
        a[t] = n < 0 ? make_float2(0.f, 0.f) : cmul(csub(E[n - ebase], c), __ldg(ds_tab + p));
        p += step;
        p = p >= ds_den ? p - ds_den : p;
    }
    if (blockIdx.x == 0)
        for (long long m = ybase + threadIdx.x; m < f_prev; m += kFdThreads)
            Y[m - ybase] = (m < 0) ? make_float2(0.f, 0.f) : Y_prev[m - ybase_prev];
    __syncthreads();
    float2 *X = stockham<false>(a, b, N, N, tw);
    float2 *Z = X == a ? b : a;
    const int half = N >> 1, q = N >> 2;
    for (int kp = threadIdx.x; kp < half; kp += kFdThreads) Z[kp] = cmul(X[kp < q ? kp : kp + half], __ldg(H + kp));
    __syncthreads();
    if (clk && threadIdx.x < 32) {   // band-edge clock correlation: Y_k conj(Y_{k - N/4}), |k - N/8| <= w
        float2 acc = make_float2(0.f, 0.f);
        for (int k = N / 8 - wbin + (int)threadIdx.x; k <= N / 8 + wbin; k += 32) {
            const float2 a = Z[k], b = Z[k + q];   // kept positions k and (k - N/4) mod N - N/2
            acc = cadd(acc, cmulc(a, b));
        }
#pragma unroll
        for (int o = 16; o; o >>= 1)
            acc = make_float2(acc.x + __shfl_xor_sync(0xffffffffu, acc.x, o), acc.y + __shfl_xor_sync(0xffffffffu, acc.y, o));
        if (threadIdx.x == 0) clk[blockIdx.x] = acc;
    }
    float2 *z = stockham<true>(Z, X, half, N, tw);
    const long long s0 = (long long)(N / 4) * blk - ybase;   // 2-sps index of the block's first output
    for (int m = threadIdx.x; m < q; m += kFdThreads) Y[s0 + m] = cscale(z[m + N / 8], gn);
}

// W32^k = e^{-2 pi i k / 32} for k = 0..15 (cos and sin of pi k / 16)
__device__ __forceinline__ float2 w32(int k)
{
    switch (k) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return make_float2(0.98078528040323043f, -0.19509032201612825f);
    case 2: return make_float2(0.92387953251128674f, -0.38268343236508978f);
    case 3: return make_float2(0.83146961230254524f, -0.55557023301960218f);
    case 4: return make_float2(0.70710678118654752f, -0.70710678118654752f);
    case 5: return make_float2(0.55557023301960218f, -0.83146961230254524f);
    case 6: return make_float2(0.38268343236508978f, -0.92387953251128674f);
    case 7: return make_float2(0.19509032201612825f, -0.98078528040323043f);
    case 8: return make_float2(0.f, -1.f);
    case 9: return make_float2(-0.19509032201612825f, -0.98078528040323043f);
    case 10: return make_float2(-0.38268343236508978f, -0.92387953251128674f);
    case 11: return make_float2(-0.55557023301960218f, -0.83146961230254524f);
    case 12: return make_float2(-0.70710678118654752f, -0.70710678118654752f);
    case 13: return make_float2(-0.83146961230254524f, -0.55557023301960218f);
    case 14: return make_float2(-0.92387953251128674f, -0.38268343236508978f);
    default: return make_float2(-0.98078528040323043f, -0.19509032201612825f);   // k = 15
    }
}

// 32-point DFT in registers, natural order in and out, unscaled: two 16-point
// DFTs over the even and odd samples and one radix-2 combination
template <bool INV>
__device__ __forceinline__ void dft32(float2 (&x)[32])
{
    float2 e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; i++) {
        e[i] = x[2 * i];
        o[i] = x[2 * i + 1];
    }
    dft16<INV>(e);
    dft16<INV>(o);
#pragma unroll
    for (int k = 0; k < 16; k++) {
        float2 w = w32(k);
        if (INV) w.y = -w.y;
        const float2 t = cmul(o[k], w);
        x[k] = cadd(e[k], t);
        x[k + 16] = csub(e[k], t);
    }
}

// The 1024-point form, one warp per block, as a 32 x 32 four-step transform with
// n = lane + 32 q and k = k2 + 32 k1:
//   forward: 32-point DFTs over q in registers, twiddle W1024^(lane k2), a padded
//     shared-memory transpose, 32-point DFTs over the former lane index: lane k2
//     then holds the bins k2 + 32 k1;
//   the kept bins (k1 < 8 or k1 >= 24) times the response give the 512-point
//     spectrum at k' = lane + 32 j (j = k1, or k1 - 16);
//   inverse with m = m_a + 16 m_b: 16-point inverse DFTs over j in registers,
//     twiddle e^{+2 pi i lane m_a / 512}, a transpose, then per m_a the inverse
//     32-point DFT over the lanes split between a lane pair (even / odd lanes,
//     16 points each, halves exchanged by shuffles), evaluated only at the kept
//     outputs m_b = 8 .. 23 (m = 128 .. 383).
constexpr int kFdWarps = 4, kFdPitch = 33;

__global__ void __launch_bounds__(32 * kFdWarps, 4)
    k_kk_fd1024(const float2 *__restrict__ E, long long ebase, long long b_first, long long nblk,
                const float2 *__restrict__ H, const float2 *__restrict__ tw, const float2 *__restrict__ ds_tab,
                int ds_num, int ds_den, const double *__restrict__ cg, float2 *__restrict__ Y, long long ybase,
                long long f_prev, const float2 *__restrict__ Y_prev, long long ybase_prev,
                float2 *__restrict__ clk, int wbin)
{
    __shared__ float2 s_tw[1024];
    __shared__ float2 s_t[kFdWarps][32 * kFdPitch];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) s_tw[i] = tw[i];
    if (blockIdx.x == 0)
        for (long long m = ybase + threadIdx.x; m < f_prev; m += blockDim.x)
            Y[m - ybase] = (m < 0) ? make_float2(0.f, 0.f) : Y_prev[m - ybase_prev];
    __syncthreads();
    const long long bi = (long long)blockIdx.x * kFdWarps + w;
    if (bi >= nblk) return;
    const long long blk = b_first + bi, n0 = 512 * blk - 256;
    const float2 c = make_float2((float)cg[0], (float)cg[1]);
    const float gn = (float)cg[2];
    long long r0 = (n0 + lane) % ds_den;
    if (r0 < 0) r0 += ds_den;
    int p = (int)((r0 * ds_num) % ds_den);
    const int step = (int)((32LL * ds_num) % ds_den);
    float2 x[32];
#pragma unroll
    for (int q = 0; q < 32; q++) {
        const long long n = n0 + lane + 32 * q;
        x[q] = n < 0 ? make_float2(0.f, 0.f) : cmul(csub(E[n - ebase], c), __ldg(ds_tab + p));
        p += step;
        p = p >= ds_den ? p - ds_den : p;
    }
    dft32<false>(x);
#pragma unroll
    for (int k2 = 1; k2 < 32; k2++) x[k2] = cmul(x[k2], s_tw[lane * k2]);
    float2 *T = s_t[w];
#pragma unroll
    for (int k2 = 0; k2 < 32; k2++) T[lane * kFdPitch + k2] = x[k2];
    __syncwarp();
#pragma unroll
    for (int n1 = 0; n1 < 32; n1++) x[n1] = T[n1 * kFdPitch + lane];
    __syncwarp();
    dft32<false>(x);
    float2 z[16];
#pragma unroll
    for (int j = 0; j < 16; j++) z[j] = cmul(x[j < 8 ? j : j + 16], __ldg(H + lane + 32 * j));
    if (clk) {   // band-edge clock correlation: bins k = lane + 32 k1 (k1 = 3, 4) with k - 256 (k1 + 24 -> j + 8)
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k1 = 3; k1 <= 4; k1++) {
            const int k = lane + 32 * k1;
            if (k >= 128 - wbin && k <= 128 + wbin) acc = cadd(acc, cmulc(z[k1], z[k1 + 8]));
        }
#pragma unroll
        for (int o = 16; o; o >>= 1)
            acc = make_float2(acc.x + __shfl_xor_sync(0xffffffffu, acc.x, o), acc.y + __shfl_xor_sync(0xffffffffu, acc.y, o));
        if (lane == 0) clk[bi] = acc;
    }
    dft16<true>(z);
#pragma unroll
    for (int ma = 1; ma < 16; ma++) z[ma] = cmulc(z[ma], s_tw[2 * lane * ma]);
#pragma unroll
    for (int ma = 0; ma < 16; ma++) T[lane * 17 + ma] = z[ma];
    __syncwarp();
    const int ma = lane >> 1, h = lane & 1;
#pragma unroll
    for (int i = 0; i < 16; i++) z[i] = T[(2 * i + h) * 17 + ma];
    dft16<true>(z);   // h = 0: even-lane half E[r]; h = 1: odd-lane half O[r]
    const long long s0 = 256 * blk - ybase;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        // lane h = 0 emits m_b = 8 + i (r = 8 + i), lane h = 1 emits m_b = 16 + i (r = i)
        const float2 send = h ? z[8 + i] : z[i];
        const float2 other = make_float2(__shfl_xor_sync(0xffffffffu, send.x, 1),
                                         __shfl_xor_sync(0xffffffffu, send.y, 1));
        const float2 Ev = h ? other : z[8 + i], Ov = h ? z[i] : other;
        float2 wv = h ? w32(i) : w32(8 + i);   // e^{+2 pi i m_b / 32} = conj(W32^r), negated for m_b >= 16
        wv.y = -wv.y;
        if (h) wv = make_float2(-wv.x, -wv.y);
        Y[s0 + ma + 16 * (8 * h + i)] = cscale(cadd(Ev, cmul(wv, Ov)), gn);
    }
}

cudaError_t launch_kk_fdmf(const float2 *E, long long ebase, long long f_prev, long long f_k, int N,
                           const float2 *H, const float2 *tw, const float2 *ds_tab, int ds_num, int ds_den,
                           const double *cg, float2 *Y, long long ybase, const float2 *Y_prev,
                           long long ybase_prev, cudaStream_t st, float2 *clk, int wbin)
{
    const int per = N / 4;   // outputs per block
    if (N < 16 || (N & (N - 1)) || f_prev % per || f_k % per || wbin < 0 || wbin >= N / 8 || (N == 1024 && wbin > 31))
        return cudaErrorInvalidValue;
    const long long nblk = (f_k - f_prev) / per;
    if (nblk <= 0) return cudaSuccess;
    if (N == 1024) {
        k_kk_fd1024<<<(unsigned)((nblk + kFdWarps - 1) / kFdWarps), 32 * kFdWarps, 0, st>>>(
            E, ebase, f_prev / per, nblk, H, tw, ds_tab, ds_num, ds_den, cg, Y, ybase, f_prev, Y_prev, ybase_prev,
            clk, wbin);
        return cudaGetLastError();
    }
    k_kk_fdmf<<<(unsigned)nblk, kFdThreads, 2 * N * sizeof(float2), st>>>(
        E, ebase, f_prev / per, N, H, tw, ds_tab, ds_num, ds_den, cg, Y, ybase, f_prev, Y_prev, ybase_prev, clk, wbin);
    return cudaGetLastError();
}

// =========================================================== PAM matched filter
// x[n] = (code[n] - mu) / sd with the buffer's exact integer moments, x[n < 0] = 0;
// y[m] = sum_i h_i x[m - i] at 2 samples/symbol.
__global__ void __launch_bounds__(kMfOut) k_pam_mf(const uint16_t *__restrict__ codes, long long cbase,
                                                  long long nb, long long n_end, long long f_prev, long long f_k,
                                                  const float *__restrict__ rrc, int hmf, DevState *dst,
                                                  int parity, float *__restrict__ Y, long long ybase,
                                                  const float *__restrict__ Y_prev, long long ybase_prev)
{
    extern __shared__ float xf[];
    __shared__ float s_mu, s_inv;
    if (threadIdx.x == 0) {
        double mu = (double)dst->pam_s1[parity] / (double)nb;
        double var = (double)dst->pam_s2[parity] / (double)nb - mu * mu;
        double inv = (var > 0.0) ? 1.0 / sqrt(var) : 1.0;
        s_mu = (float)mu;
        s_inv = (float)inv;
        if (blockIdx.x == 0) {
            dst->pam_mu = mu;
            dst->pam_inv_sd = inv;
        }
    }
    __syncthreads();
    long long m0 = f_prev + (long long)blockIdx.x * kMfOut;
    int L = kMfOut + 2 * hmf;
    long long n0 = m0 - hmf;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        long long n = n0 + i;
        float v = 0.f;
        if (n >= 0 && n < n_end) v = ((float)codes[n - cbase] - s_mu) * s_inv;
        xf[i] = v;
    }
    if (blockIdx.x == 0) {
        for (long long m = ybase + threadIdx.x; m < f_prev; m += blockDim.x)
            Y[m - ybase] = (m < 0) ? 0.f : Y_prev[m - ybase_prev];
        if (threadIdx.x == 0) {   // the sums of the call after next start from zero
            dst->pam_s1[(parity + 2) % 3] = 0;
            dst->pam_s2[(parity + 2) % 3] = 0;
        }
    }
    __syncthreads();
    long long m = m0 + threadIdx.x;
    if (m >= f_k) return;
    const float *xc = xf + threadIdx.x + hmf;
    float a = 0.f;
    for (int i = -hmf; i <= hmf; i++) a = fmaf(__ldg(rrc + i + hmf), xc[-i], a);
    Y[m - ybase] = a;
}

// ========================================== PAM resampler path (ADC off the transmitter's clock)
// The normalised code x[n] = (code - mu) / sd of the call (complex, imaginary part 0)
// for stream samples [cbase, n_end), the input of the resampler (which treats
// samples before the stream as zero); the call's mean and deviation come from the
// exact integer sums, and the sums of the next call start from zero.
__global__ void k_pam_norm(const uint16_t *__restrict__ codes, long long cbase, long long nb, long long n_end,
                           DevState *dst, int parity, float2 *__restrict__ X)
{
    __shared__ float s_mu, s_inv;
    if (threadIdx.x == 0) {
        double mu = (double)dst->pam_s1[parity] / (double)nb;
        double var = (double)dst->pam_s2[parity] / (double)nb - mu * mu;
        double inv = (var > 0.0) ? 1.0 / sqrt(var) : 1.0;
        s_mu = (float)mu;
        s_inv = (float)inv;
    }
    __syncthreads();
    const long long n = cbase + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n < n_end) X[n - cbase] = make_float2(((float)codes[n - cbase] - s_mu) * s_inv, 0.f);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        dst->pam_mu = (double)s_mu;
        dst->pam_inv_sd = (double)s_inv;
        dst->pam_s1[(parity + 2) % 3] = 0;   // the sums of the call after next start from zero
        dst->pam_s2[(parity + 2) % 3] = 0;
    }
}

// the PAM matched filter (2 samples/symbol, no decimation) on the resampled series
// (real parts of R, stream index m at R[m - rbase]; zero before the stream)
__global__ void __launch_bounds__(kMfOut) k_pam_mf_r(const float2 *__restrict__ R, long long rbase, long long f_prev,
                                                    long long f_k, const float *__restrict__ rrc, int hmf,
                                                    float *__restrict__ Y, long long ybase,
                                                    const float *__restrict__ Y_prev, long long ybase_prev)
{
    extern __shared__ float xf[];
    long long m0 = f_prev + (long long)blockIdx.x * kMfOut;
    int L = kMfOut + 2 * hmf;
    long long n0 = m0 - hmf;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        long long n = n0 + i;
        xf[i] = n < 0 ? 0.f : R[n - rbase].x;
    }
    if (blockIdx.x == 0)
        for (long long m = ybase + threadIdx.x; m < f_prev; m += blockDim.x)
            Y[m - ybase] = (m < 0) ? 0.f : Y_prev[m - ybase_prev];
    __syncthreads();
    long long m = m0 + threadIdx.x;
    if (m >= f_k) return;
    const float *xc = xf + threadIdx.x + hmf;
    float a = 0.f;
    for (int i = -hmf; i <= hmf; i++) a = fmaf(__ldg(rrc + i + hmf), xc[-i], a);
    Y[m - ybase] = a;
}

cudaError_t launch_pam_norm(const uint16_t *codes, long long cbase, long long nb, long long n_end, DevState *dst,
                            int parity, float2 *X, cudaStream_t st)
{
    const long long n = n_end - cbase;
    k_pam_norm<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(codes, cbase, nb, n_end, dst, parity, X);
    return cudaGetLastError();
}

cudaError_t launch_pam_mf_r(const float2 *R, long long rbase, long long f_prev, long long f_k, const float *rrc, int hmf,
                            float *Y, long long ybase, const float *Y_prev, long long ybase_prev, cudaStream_t st)
{
    long long n = f_k - f_prev;
    unsigned grid = (unsigned)((n + kMfOut - 1) / kMfOut);
    size_t smem = (size_t)(kMfOut + 2 * hmf) * sizeof(float);
    k_pam_mf_r<<<grid, kMfOut, smem, st>>>(R, rbase, f_prev, f_k, rrc, hmf, Y, ybase, Y_prev, ybase_prev);
    return cudaGetLastError();
}

// ===================================================== PAM frequency-domain filter
// The paper's PAM form (Sec. 2): a static filter applied on 1024-point
// overlap-save blocks (hop 512) at the input rate.  One warp per block: the
// normalised codes x[n] = (code - mu) / sd of the N inputs from 512 b - 256 go
// through the same 32 x 32 four-step forward transform as the KK form (lane k2
// holds the bins k2 + 32 k1), every bin is multiplied by the response (times
// 1/N), and the 1024-point inverse runs as a second four-step with m = m_a + 32
// m_b: 32-point inverse DFTs over k1 in registers, twiddle e^{+2 pi i lane m_a /
// 1024}, a transpose, 32-point inverse DFTs over the former lane index; lane m_a
// keeps m_b = 8 .. 23 (m = 256 .. 767), whose real part is y.
__global__ void __launch_bounds__(32 * kFdWarps, 4)
    k_pam_fd1024(const uint16_t *__restrict__ codes, long long cbase, long long nb, long long n_end,
                 long long b_first, long long nblk, const float2 *__restrict__ H, const float2 *__restrict__ tw,
                 DevState *dst, int parity, float *__restrict__ Y, long long ybase, long long f_prev,
                 const float *__restrict__ Y_prev, long long ybase_prev, float2 *__restrict__ clk, int wbin)
{
    __shared__ float2 s_tw[1024];
    __shared__ float2 s_t[kFdWarps][32 * kFdPitch];
    __shared__ float s_mu, s_inv;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) s_tw[i] = tw[i];
    if (threadIdx.x == 0) {
        double mu = (double)dst->pam_s1[parity] / (double)nb;
        double var = (double)dst->pam_s2[parity] / (double)nb - mu * mu;
        double inv = (var > 0.0) ? 1.0 / sqrt(var) : 1.0;
        s_mu = (float)mu;
        s_inv = (float)inv;
    }
    __syncthreads();
    if (blockIdx.x == 0) {
        for (long long m = ybase + threadIdx.x; m < f_prev; m += blockDim.x)
            Y[m - ybase] = (m < 0) ? 0.f : Y_prev[m - ybase_prev];
        if (threadIdx.x == 0) {   // debug view; the sums of the next call start from zero
            double mu = (double)dst->pam_s1[parity] / (double)nb;
            double var = (double)dst->pam_s2[parity] / (double)nb - mu * mu;
            dst->pam_mu = mu;
            dst->pam_inv_sd = (var > 0.0) ? 1.0 / sqrt(var) : 1.0;
            dst->pam_s1[(parity + 2) % 3] = 0;
            dst->pam_s2[(parity + 2) % 3] = 0;
        }
    }
    const long long bi = (long long)blockIdx.x * kFdWarps + w;
    if (bi >= nblk) return;
    const long long blk = b_first + bi, n0 = 512 * blk - 256;
    const float mu = s_mu, inv = s_inv;
    float2 x[32];
#pragma unroll
    for (int q = 0; q < 32; q++) {
        const long long n = n0 + lane + 32 * q;
        x[q] = make_float2(n >= 0 && n < n_end ? ((float)codes[n - cbase] - mu) * inv : 0.f, 0.f);
    }
    dft32<false>(x);
#pragma unroll
    for (int k2 = 1; k2 < 32; k2++) x[k2] = cmul(x[k2], s_tw[lane * k2]);
    float2 *T = s_t[w];
#pragma unroll
    for (int k2 = 0; k2 < 32; k2++) T[lane * kFdPitch + k2] = x[k2];
    __syncwarp();
#pragma unroll
    for (int n1 = 0; n1 < 32; n1++) x[n1] = T[n1 * kFdPitch + lane];
    __syncwarp();
    dft32<false>(x);   // x[k1] = X[lane + 32 k1]
#pragma unroll
    for (int k1 = 0; k1 < 32; k1++) x[k1] = cmul(x[k1], __ldg(H + lane + 32 * k1));
    if (clk) {   // band-edge clock correlation at 2 samples/symbol: bins k = lane + 32 k1 (k1 = 7, 8)
                 // around N/4 with k - N/2 (k1 + 16)
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k1 = 7; k1 <= 8; k1++) {
            const int k = lane + 32 * k1;
            if (k >= 256 - wbin && k <= 256 + wbin) acc = cadd(acc, cmulc(x[k1], x[k1 + 16]));
        }
#pragma unroll
        for (int o = 16; o; o >>= 1)
            acc = make_float2(acc.x + __shfl_xor_sync(0xffffffffu, acc.x, o), acc.y + __shfl_xor_sync(0xffffffffu, acc.y, o));
        if (lane == 0) clk[bi] = acc;
    }
    dft32<true>(x);    // over k1 -> m_a
#pragma unroll
    for (int ma = 1; ma < 32; ma++) x[ma] = cmulc(x[ma], s_tw[lane * ma]);
#pragma unroll
    for (int ma = 0; ma < 32; ma++) T[lane * kFdPitch + ma] = x[ma];
    __syncwarp();
#pragma unroll
    for (int l = 0; l < 32; l++) x[l] = T[l * kFdPitch + lane];
    dft32<true>(x);    // lane m_a: x[m_b] = z[m_a + 32 m_b]
    const long long s0 = 512 * blk - ybase;
#pragma unroll
    for (int mb = 8; mb < 24; mb++) Y[s0 + lane + 32 * (mb - 8)] = x[mb].x;
}

cudaError_t launch_pam_fd1024(const uint16_t *codes, long long cbase, long long nb, long long n_end,
                              long long f_prev, long long f_k, const float2 *H, const float2 *tw, DevState *dst,
                              int parity, float *Y, long long ybase, const float *Y_prev, long long ybase_prev,
                              cudaStream_t st, float2 *clk, int wbin)
{
    if (f_prev % 512 || f_k % 512 || wbin < 0 || wbin > 31) return cudaErrorInvalidValue;
    const long long nblk = (f_k - f_prev) / 512;
    if (nblk <= 0) return cudaSuccess;
    k_pam_fd1024<<<(unsigned)((nblk + kFdWarps - 1) / kFdWarps), 32 * kFdWarps, 0, st>>>(
        codes, cbase, nb, n_end, f_prev / 512, nblk, H, tw, dst, parity, Y, ybase, f_prev, Y_prev, ybase_prev, clk,
        wbin);
    return cudaGetLastError();
}

// Register-tiled PAM matched filter for a compile-time half length HMF: each thread
// computes kPmR consecutive outputs from a sliding window held in registers (one
// shared-memory load per tap), the taps read from shared memory as broadcasts.  Per
// output the products are accumulated in the same order as k_pam_mf (tap index
// ascending), so the outputs are the same bit for bit.
constexpr int kPmThreads = 128, kPmR = 8, kPmTile = kPmThreads * kPmR;

template <int HMF>
__global__ void __launch_bounds__(kPmThreads) k_pam_mf_t(const uint16_t *__restrict__ codes, long long cbase,
                                                        long long nb, long long n_end, long long f_prev, long long f_k,
                                                        const float *__restrict__ rrc, DevState *dst, int parity,
                                                        float *__restrict__ Y, long long ybase,
                                                        const float *__restrict__ Y_prev, long long ybase_prev)
{
    __shared__ float xf[kPmTile + 2 * HMF];
    __shared__ float s_h[2 * HMF + 1];
    __shared__ float s_mu, s_inv;
    if (threadIdx.x == 0) {
        double mu = (double)dst->pam_s1[parity] / (double)nb;
        double var = (double)dst->pam_s2[parity] / (double)nb - mu * mu;
        double inv = (var > 0.0) ? 1.0 / sqrt(var) : 1.0;
        s_mu = (float)mu;
        s_inv = (float)inv;
        if (blockIdx.x == 0) {
            dst->pam_mu = mu;
            dst->pam_inv_sd = inv;
        }
    }
    for (int i = threadIdx.x; i <= 2 * HMF; i += kPmThreads) s_h[i] = __ldg(rrc + i);
    __syncthreads();
    const long long m0 = f_prev + (long long)blockIdx.x * kPmTile;
    const long long n0 = m0 - HMF;
    const float mu = s_mu, inv = s_inv;
    for (int i = threadIdx.x; i < kPmTile + 2 * HMF; i += kPmThreads) {
        const long long n = n0 + i;
        xf[i] = (n >= 0 && n < n_end) ? ((float)codes[n - cbase] - mu) * inv : 0.f;
    }
    if (blockIdx.x == 0) {
        for (long long m = ybase + threadIdx.x; m < f_prev; m += blockDim.x)
            Y[m - ybase] = (m < 0) ? 0.f : Y_prev[m - ybase_prev];
        if (threadIdx.x == 0) {   // the sums of the call after next start from zero
            dst->pam_s1[(parity + 2) % 3] = 0;
            dst->pam_s2[(parity + 2) % 3] = 0;
        }
    }
    __syncthreads();
    // output j = j0 + r: y = sum_{i=-HMF}^{HMF} h[i + HMF] xf[j + HMF - i]; with u = HMF - i
    // running from 2 HMF down to 0 the window xf[j0 + u + r] slides down by one per tap
    const int j0 = kPmR * threadIdx.x;
    float win[kPmR], acc[kPmR];
#pragma unroll
    for (int r = 0; r < kPmR; r++) {
        win[r] = xf[j0 + 2 * HMF + r];
        acc[r] = 0.f;
    }
#pragma unroll
    for (int u = 2 * HMF; u >= 0; u--) {
        const float hu = s_h[2 * HMF - u];
#pragma unroll
        for (int r = 0; r < kPmR; r++) acc[r] = fmaf(hu, win[r], acc[r]);
        if (u > 0) {
#pragma unroll
            for (int r = kPmR - 1; r > 0; r--) win[r] = win[r - 1];
            win[0] = xf[j0 + u - 1];
        }
    }
    const long long mb = m0 + j0;
#pragma unroll
    for (int r = 0; r < kPmR; r++)
        if (mb + r < f_k) Y[mb + r - ybase] = acc[r];
}

cudaError_t launch_pam_mf(const uint16_t *codes, long long cbase, long long nb, long long n_end, long long f_prev,
                          long long f_k, const float *rrc, int hmf, DevState *dst, int parity,
                          float *Y, long long ybase, const float *Y_prev, long long ybase_prev,
                          cudaStream_t st)
{
    long long n = f_k - f_prev;
    if (hmf == 16) {   // the default span (16 symbols at 2 samples/symbol)
        unsigned grid = (unsigned)((n + kPmTile - 1) / kPmTile);
        k_pam_mf_t<16><<<grid, kPmThreads, 0, st>>>(codes, cbase, nb, n_end, f_prev, f_k, rrc, dst, parity, Y, ybase,
                                                    Y_prev, ybase_prev);
        return cudaGetLastError();
    }
    unsigned grid = (unsigned)((n + kMfOut - 1) / kMfOut);
    size_t smem = (size_t)(kMfOut + 2 * hmf) * sizeof(float);
    k_pam_mf<<<grid, kMfOut, smem, st>>>(codes, cbase, nb, n_end, f_prev, f_k, rrc, hmf, dst, parity, Y,
                                         ybase, Y_prev, ybase_prev);
    return cudaGetLastError();
}

// bin and clear every latency slot still holding a record (rx_stats)
__global__ void k_lat_flush(LatRecord *r)
{
    const int i = threadIdx.x;
    if (i < kLatSlots) {
        const unsigned long long t0 = r->slot[i].t0, t1 = r->slot[i].t1;
        r->slot[i].t0 = 0ull;
        r->slot[i].t1 = 0ull;
        lat_bin(r, t0, t1);
    }
}

cudaError_t launch_lat_flush(LatRecord *r, cudaStream_t st)
{
    k_lat_flush<<<1, kLatSlots, 0, st>>>(r);
    return cudaGetLastError();
}

}  // namespace rxk
