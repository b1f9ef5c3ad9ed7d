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
                         long long *s2)
{
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
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
                          int pack_order, long long *s1, long long *s2, cudaStream_t st)
{
    long long items = nb / 8 + nhist;
    int tpb = 256;
    unsigned grid = (unsigned)((items + tpb - 1) / tpb);
    k_unpack<<<grid, tpb, 0, st>>>(in, codes, codes_prev, nb, nhist, prev_off, first_call,
                                   pack_order, s1, s2);
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
// and only keeps the FP32 FFT well scaled); I = code, 0.5 for code 0
__device__ __forceinline__ float kk_u(uint16_t code)
{
    float I = code ? (float)code : 0.5f;
    return 0.5f * logf(I * (1.0f / 2048.0f));
}

// K1a: radix-16 pass over the stride-N2 index of two packed blocks, then twiddle.
__global__ void __launch_bounds__(kCtaK1) k_kk_fwd(KkGeom g, const uint16_t *__restrict__ codes,
                                                  float2 *__restrict__ fftws, const float2 *__restrict__ twN)
{
    int pair = blockIdx.y;
    int n1 = blockIdx.x * blockDim.x + threadIdx.x;
    if (n1 >= g.N2) return;
    int ja = 2 * pair, jb = 2 * pair + 1;
    long long oa = ols_ws(g, ja) - g.cbase;
    bool hb = jb < g.J;
    long long ob = hb ? ols_ws(g, jb) - g.cbase : 0;
    float2 x[16];
#pragma unroll
    for (int q = 0; q < 16; q++) {
        long long t = n1 + (long long)g.N2 * q;
        float ua = kk_u(__ldg(codes + oa + t));
        float ub = hb ? kk_u(__ldg(codes + ob + t)) : 0.f;
        x[q] = make_float2(ua, ub);
    }
    dft16<false>(x);
    float2 *out = fftws + (size_t)pair * g.N + n1;
#pragma unroll
    for (int k2 = 0; k2 < 16; k2++) {
        float2 w = __ldg(twN + n1 * k2);
        out[(size_t)k2 * g.N2] = cmul(x[k2], w);
    }
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
__global__ void __launch_bounds__(256) k_kk_rows(KkGeom g, float2 *__restrict__ fftws,
                                                const float2 *__restrict__ twN2)
{
    constexpr int N2 = 1 << (4 * P);
    constexpr int TPR = N2 / 16;                  // threads per row
    constexpr int RPC = 256 / TPR;                // rows per CTA
    constexpr int SROW = N2 + N2 / 16;            // padded row in shared memory
    extern __shared__ float2 sm[];
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
#pragma unroll
    for (int r = 1; r < 16; r++) x[r] = cmul(x[r], __ldg(twN2 + ((t * r) & (N2 - 1))));
    if (P == 1) {
#pragma unroll
        for (int r = 0; r < 16; r++) x[r] = hilbert_mul(x[r], k2 + 16 * drev16<P>(r), g.N);
        dft16<true>(x);
        if (active)
#pragma unroll
            for (int r = 0; r < 16; r++) d[r] = x[r];
        return;
    }
#pragma unroll
    for (int r = 0; r < 16; r++) s[pad16(t + r * TPR)] = x[r];
    __syncthreads();
    // remaining forward passes; the last one is fused with the multiplier and the
    // first inverse pass
#pragma unroll
    for (int p = 1; p < P; p++) {
        const int M = N2 >> (4 * p), sub = M / 16;
        int o = (t / sub) * M, j = t % sub;
#pragma unroll
        for (int r = 0; r < 16; r++) x[r] = s[pad16(o + j + r * sub)];
        dft16<false>(x);
        if (p < P - 1) {
#pragma unroll
            for (int r = 1; r < 16; r++) x[r] = cmul(x[r], __ldg(twN2 + ((j * r * (N2 / M)) & (N2 - 1))));
#pragma unroll
            for (int r = 0; r < 16; r++) s[pad16(o + j + r * sub)] = x[r];
            __syncthreads();
        } else {
            // M = 16: positions o + r hold X[k2 + 16 * drev(o + r)]
#pragma unroll
            for (int r = 0; r < 16; r++) x[r] = hilbert_mul(x[r], k2 + 16 * drev16<P>(o + r), g.N);
            dft16<true>(x);
#pragma unroll
            for (int r = 0; r < 16; r++) s[pad16(o + r)] = x[r];
            __syncthreads();
        }
    }
    // inverse passes P-2 .. 1
#pragma unroll
    for (int p = P - 2; p >= 1; p--) {
        const int M = N2 >> (4 * p), sub = M / 16;
        int o = (t / sub) * M, j = t % sub;
#pragma unroll
        for (int r = 0; r < 16; r++) {
            x[r] = s[pad16(o + j + r * sub)];
            if (r) x[r] = cmulc(x[r], __ldg(twN2 + ((j * r * (N2 / M)) & (N2 - 1))));
        }
        dft16<true>(x);
#pragma unroll
        for (int r = 0; r < 16; r++) s[pad16(o + j + r * sub)] = x[r];
        __syncthreads();
    }
    // inverse pass 0 to global memory
#pragma unroll
    for (int r = 0; r < 16; r++) {
        x[r] = s[pad16(t + r * TPR)];
        if (r) x[r] = cmulc(x[r], __ldg(twN2 + ((t * r) & (N2 - 1))));
    }
    dft16<true>(x);
    if (active)
#pragma unroll
        for (int r = 0; r < 16; r++) d[t + r * TPR] = x[r];
}

// K1c: inverse radix-16 pass, then for every kept output
// E = sqrt(I) * exp(j phi) (Fig. 1d), written at its stream position, and the
// per-call carrier / intensity sums (deterministic: fixed-order trees, last-CTA
// finalisation in FP64).
__global__ void __launch_bounds__(kCtaK1) k_kk_inv(KkGeom g, const uint16_t *__restrict__ codes,
                                                  const float2 *__restrict__ fftws,
                                                  const float2 *__restrict__ twN, float2 *__restrict__ E,
                                                  const float2 *__restrict__ E_prev,
                                                  CarrierPartial *__restrict__ partials, DevState *dst)
{
    int pair = blockIdx.y;
    int n1 = blockIdx.x * blockDim.x + threadIdx.x;
    float sre = 0.f, sim = 0.f;
    int si2 = 0;
    if (blockIdx.x == 0 && blockIdx.y == 0) {
        // field history for the matched filter: E[n], n in [e_prev - kEHist, e_prev)
        for (int i = threadIdx.x; i < kEHist; i += blockDim.x) {
            long long n = g.e_prev - kEHist + i;
            E[i] = (n < 0) ? make_float2(0.f, 0.f) : E_prev[n - g.ebase_prev];
        }
    }
    if (n1 < g.N2) {
        float2 x[16];
        const float2 *in = fftws + (size_t)pair * g.N + n1;
#pragma unroll
        for (int k2 = 0; k2 < 16; k2++) x[k2] = cmulc(in[(size_t)k2 * g.N2], __ldg(twN + n1 * k2));
        dft16<true>(x);
        const float invN = 1.0f / (float)g.N;
#pragma unroll
        for (int half = 0; half < 2; half++) {
            int j = 2 * pair + half;
            if (j >= g.J) break;
            long long ws = ols_ws(g, j);
            int tlo, thi;
            ols_kept(g, j, tlo, thi);
#pragma unroll
            for (int q = 0; q < 16; q++) {
                int t = n1 + g.N2 * q;
                if (t < tlo || t >= thi) continue;
                long long n = ws + t;
                uint16_t code = __ldg(codes + (n - g.cbase));
                float I = code ? (float)code : 0.5f;
                float phi = (half ? x[q].y : x[q].x) * invN;
                float sn, cs;
                sincosf(phi, &sn, &cs);
                float A = sqrtf(I);
                float2 e = make_float2(A * cs, A * sn);
                E[n - g.ebase] = e;
                sre += e.x;
                sim += e.y;
                si2 += code ? 2 * (int)code : 1;
            }
        }
    }
    // CTA partial (fixed-order tree)
    __shared__ float rre[kCtaK1 / 32], rim[kCtaK1 / 32];
    __shared__ int ri[kCtaK1 / 32];
    __shared__ bool last;
    sre = warp_sum_f(sre);
    sim = warp_sum_f(sim);
    si2 = warp_sum_i(si2);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { rre[wid] = sre; rim[wid] = sim; ri[wid] = si2; }
    __syncthreads();
    int cta = blockIdx.y * gridDim.x + blockIdx.x;
    int ncta = gridDim.x * gridDim.y;
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        long long c = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) { a += rre[i]; b += rim[i]; c += ri[i]; }
        partials[cta].re = a;
        partials[cta].im = b;
        partials[cta].i2 = c;
        __threadfence();
        unsigned tk = atomicAdd(&dst->ticket, 1u);
        last = (tk == (unsigned)(ncta - 1));
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // last CTA: strided per-thread sums then a fixed-order tree in FP64
    __shared__ double dre[kCtaK1], dim[kCtaK1];
    __shared__ long long dii[kCtaK1];
    double a = 0, b = 0;
    long long c = 0;
    for (int i = threadIdx.x; i < ncta; i += blockDim.x) {
        volatile CarrierPartial *pp = partials + i;
        a += pp->re;
        b += pp->im;
        c += pp->i2;
    }
    dre[threadIdx.x] = a;
    dim[threadIdx.x] = b;
    dii[threadIdx.x] = c;
    __syncthreads();
    for (int sft = blockDim.x / 2; sft > 0; sft >>= 1) {
        if ((int)threadIdx.x < sft) {
            dre[threadIdx.x] += dre[threadIdx.x + sft];
            dim[threadIdx.x] += dim[threadIdx.x + sft];
            dii[threadIdx.x] += dii[threadIdx.x + sft];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double cnt = (double)(g.e_k - g.e_prev);
        double cr = dre[0] / cnt, ci = dim[0] / cnt;
        double ibar = (double)dii[0] / (2.0 * cnt);
        double P = ibar - (cr * cr + ci * ci);
        dst->carrier_re = cr;
        dst->carrier_im = ci;
        dst->gain = (P > 0.0) ? 1.0 / sqrt((double)g.sps * P) : 1.0;
        dst->ticket = 0u;
    }
}

cudaError_t launch_kk_front(const KkGeom &g, const uint16_t *codes, float2 *fftws,
                            const float2 *twN, const float2 *twN2, float2 *E, const float2 *E_prev,
                            CarrierPartial *partials, DevState *dst, cudaStream_t st, void *prof)
{
    dim3 grid((g.N2 + kCtaK1 - 1) / kCtaK1, g.npairs);
    prof_stage(prof, 1, st);
    k_kk_fwd<<<grid, kCtaK1, 0, st>>>(g, codes, fftws, twN);
    prof_stage(prof, 2, st);
    int rows = g.npairs * 16;
    if (g.N2 == 4096) {
        size_t smem = (size_t)(4096 + 256) * sizeof(float2);
        k_kk_rows<3><<<rows, 256, smem, st>>>(g, fftws, twN2);
    } else if (g.N2 == 256) {
        size_t smem = (size_t)16 * (256 + 16) * sizeof(float2);
        k_kk_rows<2><<<(rows + 15) / 16, 256, smem, st>>>(g, fftws, twN2);
    } else {
        k_kk_rows<1><<<(rows + 255) / 256, 256, 0, st>>>(g, fftws, twN2);
    }
    prof_stage(prof, 3, st);
    k_kk_inv<<<grid, kCtaK1, 0, st>>>(g, codes, fftws, twN, E, E_prev, partials, dst);
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
                                                 int ds_den, const DevState *__restrict__ dst,
                                                 float2 *__restrict__ Y, long long ybase,
                                                 const float2 *__restrict__ Y_prev, long long ybase_prev)
{
    extern __shared__ float2 xs[];
    long long m0 = f_prev + (long long)blockIdx.x * kMfOut;
    int L = 2 * kMfOut + 2 * hmf;
    float2 c = make_float2((float)dst->carrier_re, (float)dst->carrier_im);
    float gn = (float)dst->gain;
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

cudaError_t launch_kk_mf(const float2 *E, long long ebase, long long e_k, long long f_prev,
                         long long f_k, const float *rrc, int hmf, const float2 *ds_tab,
                         int ds_num, int ds_den, const DevState *dst, float2 *Y, long long ybase,
                         const float2 *Y_prev, long long ybase_prev, cudaStream_t st)
{
    long long n = f_k - f_prev;
    unsigned grid = (unsigned)((n + kMfOut - 1) / kMfOut);
    size_t smem = (size_t)(2 * kMfOut + 2 * hmf) * sizeof(float2);
    k_kk_mf<<<grid, kMfOut, smem, st>>>(E, ebase, e_k, f_prev, f_k, rrc, hmf, ds_tab, ds_num,
                                        ds_den, dst, Y, ybase, Y_prev, ybase_prev);
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
        if (threadIdx.x == 0) {   // the sums of the next call start from zero
            dst->pam_s1[parity ^ 1] = 0;
            dst->pam_s2[parity ^ 1] = 0;
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

cudaError_t launch_pam_mf(const uint16_t *codes, long long cbase, long long nb, long long n_end, long long f_prev,
                          long long f_k, const float *rrc, int hmf, DevState *dst, int parity,
                          float *Y, long long ybase, const float *Y_prev, long long ybase_prev,
                          cudaStream_t st)
{
    long long n = f_k - f_prev;
    unsigned grid = (unsigned)((n + kMfOut - 1) / kMfOut);
    size_t smem = (size_t)(kMfOut + 2 * hmf) * sizeof(float);
    k_pam_mf<<<grid, kMfOut, smem, st>>>(codes, cbase, nb, n_end, f_prev, f_k, rrc, hmf, dst, parity, Y,
                                         ybase, Y_prev, ybase_prev);
    return cudaGetLastError();
}

}  // namespace rxk
