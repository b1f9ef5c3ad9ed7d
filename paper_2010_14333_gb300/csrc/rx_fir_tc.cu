// Block-Toeplitz FIR on the fifth-generation tensor cores (tcgen05).
//
// The equaliser's filter z_k = sum_i conj(w_i) y[2k + TH - i] with taps that are
// fixed for a whole call (the frozen form) is one dense contraction: rows of 16
// consecutive symbols, each row an (M = 1) x (K = 2 * (30 + NT) real inputs,
// padded to 128) slice of the 2-sps sequence (a Hankel matrix of y, complex
// interleaved as stored), times a K x 32 real Toeplitz matrix built from the
// taps (complex split to real:  [re; im] outputs of each symbol).  One CTA
// computes 128 rows (2048 symbols) with M = 128, N = 32 tcgen05.mma in BF16,
// FP16 or FP8-E4M3 with FP32 accumulation in tensor memory:
//   - one bulk copy (cp.async.bulk) stages the tile's 4.1 k complex inputs in
//     shared memory as FP32;
//   - the threads convert them into the K-major operand layout (core matrices
//     of 8 rows x 16 bytes; FP8 with a power-of-two scale per block of
//     rows_per_scale rows, taken from the block's largest input);
//   - one thread issues the MMAs and commits them to an mbarrier;
//   - each warp reads its 32 accumulator lanes (tcgen05.ld), rescales, stores z.
// Every wait is bounded: on time-out the kernel records RX_ETIMEOUT, waits
// (bounded) for its own copies and MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "rx_async.cuh"
#include "rx_internal.cuh"

namespace rxk {
namespace {

constexpr int kRowSyms = 16;                       // symbols per GEMM row
constexpr int kTileRows = 128;                     // M of one MMA
constexpr int kN = 2 * kRowSyms;                   // real outputs per row
constexpr int kKP = 128;                           // padded K (2 * (30 + NT) <= 122)
constexpr int kThreads = 128;
constexpr int kStage = 2 * kRowSyms * kTileRows + 64;   // staged complex inputs per tile
constexpr uint32_t kTmemCols = 32;
// dynamic shared memory: A | B | stage | barriers and scratch, padded so that a
// tile's operand reads stay inside the allocation for any stride of the layout
constexpr int kOffA = 0;
constexpr int kOffB = kOffA + kTileRows * kKP * 2;   // 32 KB (room for 16-bit A)
constexpr int kOffStage = kOffB + kN * kKP * 2;      // + 8 KB
constexpr int kOffMisc = kOffStage + kStage * 8;
constexpr int kSmem = 112 * 1024;
static_assert(kOffMisc + 1024 <= kSmem, "shared-memory plan");

template <int PREC> struct Fmt;
template <> struct Fmt<RX_FIR_BF16> {
    static constexpr int esize = 2;
    static constexpr uint32_t code = 1;   // kind::f16, BF16
};
template <> struct Fmt<RX_FIR_FP16> {
    static constexpr int esize = 2;
    static constexpr uint32_t code = 0;   // kind::f16, F16
};
template <> struct Fmt<RX_FIR_FP8> {
    static constexpr int esize = 1;
    static constexpr uint32_t code = 0;   // kind::f8f6f4, E4M3
};

// 8 (16-bit) or 16 (FP8) consecutive K elements -> one 16-byte core-matrix row
template <int PREC>
__device__ __forceinline__ uint4 pack16(const float *v, float s);
template <>
__device__ __forceinline__ uint4 pack16<RX_FIR_BF16>(const float *v, float)
{
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<uint32_t *>(&h);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}
template <>
__device__ __forceinline__ uint4 pack16<RX_FIR_FP16>(const float *v, float)
{
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        __half2 h = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<uint32_t *>(&h);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}
template <>
__device__ __forceinline__ uint4 pack16<RX_FIR_FP8>(const float *v, float s)
{
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v[4 * i] * s, v[4 * i + 1] * s), __NV_SATFINITE, __NV_E4M3);
        uint32_t hi =
            __nv_cvt_float2_to_fp8x2(make_float2(v[4 * i + 2] * s, v[4 * i + 3] * s), __NV_SATFINITE, __NV_E4M3);
        w[i] = (lo & 0xFFFFu) | (hi << 16);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// power-of-two scale that brings the largest magnitude m to at most 448 (E4M3 max)
__device__ __forceinline__ int fp8_exp(float m)
{
    if (!(m > 0.f)) return 0;
    int e;
    frexpf(448.f / m, &e);   // 448/m = f 2^e, f in [0.5, 1)
    return min(max(e - 1, -60), 60);
}

template <int PREC>
__global__ void __launch_bounds__(kThreads)
    k_fir_tc(const float2 *__restrict__ Y, long long ybase, long long k_lo, int nrows,
             const float2 *__restrict__ taps, int ntaps, int rows_per_scale, float2 *__restrict__ z, int *err)
{
    constexpr int ES = Fmt<PREC>::esize;
    constexpr int EPP = 16 / ES;                    // K elements per 16-byte core row
    constexpr int PLANES = kKP / EPP;               // K core-matrix columns
    constexpr int PLANE_A = kTileRows * 16, PLANE_B = kN * 16;
    constexpr int NMMA = PLANES / 2;                // each MMA consumes two K core matrices
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sA = sm + kOffA, *sB = sm + kOffB;
    float2 *stage = reinterpret_cast<float2 *>(sm + kOffStage);
    uint64_t *bar_ld = reinterpret_cast<uint64_t *>(sm + kOffMisc);
    uint64_t *bar_mma = bar_ld + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_ld + 2);
    int *s_exp = reinterpret_cast<int *>(sm + kOffMisc + 64);      // per scale block of the tile (<= 128)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int th = (ntaps - 1) / 2;
    const int ns = 2 * kRowSyms - 2 + ntaps;       // complex inputs per row
    const int r0 = blockIdx.x * kTileRows;
    const int rows = min(kTileRows, nrows - r0);

    // first input of the tile (stream index 2 k - TH of its first symbol), staged
    // from an even element offset so that the bulk copy starts on 16 bytes
    const long long m0 = 2 * (k_lo + (long long)r0 * kRowSyms) - th;
    const long long e0 = m0 - ybase;
    const long long es = e0 & ~1LL;
    const int shift = (int)(e0 - es);
    const int nst = ((shift + 2 * kRowSyms * (rows - 1) + ns) + 1) & ~1;   // complex inputs, even

    if (tid == 0) {
        mbar_init(bar_ld, 1);
        mbar_init(bar_mma, 1);
        mbar_expect_tx(bar_ld, (unsigned)(nst * 8));
        bulk_g2s(stage, Y + es, (unsigned)(nst * 8), bar_ld);
    }
    __syncwarp();
    if (warp == 0) tmem_alloc(tslot, kTmemCols);

    // B: Toeplitz matrix of the taps, rows n = 2j + c (c: re / im output of
    // symbol j), K index 2s + d (d: re / im of input s); tap i = 2j + 2TH - s
    float wmax = 0.f;
    for (int i = 0; i < ntaps; i++) wmax = fmaxf(wmax, fmaxf(fabsf(taps[i].x), fabsf(taps[i].y)));
    const int eB = PREC == RX_FIR_FP8 ? fp8_exp(wmax) : 0;
    const float sBv = ldexpf(1.f, eB);
    for (int u = tid; u < kN * PLANES; u += kThreads) {
        int n = u % kN, pl = u / kN;
        int j = n >> 1, c = n & 1;
        float v[16];
#pragma unroll
        for (int t = 0; t < EPP; t++) {
            int k = pl * EPP + t, s = k >> 1, d = k & 1;
            int i = 2 * j + 2 * th - s;
            float val = 0.f;
            if (s < ns && i >= 0 && i < ntaps) {
                float2 w = taps[i];
                // conj(w) y: re = a yr + b yi, im = a yi - b yr
                val = c == 0 ? (d == 0 ? w.x : w.y) : (d == 0 ? -w.y : w.x);
            }
            v[t] = val;
        }
        *reinterpret_cast<uint4 *>(sB + pl * PLANE_B + n * 16) = pack16<PREC>(v, sBv);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    bool ok = mbar_wait(bar_ld, 0);
    if (!ok) {
        atomicExch(err, (int)RX_ETIMEOUT);
        mbar_wait(bar_ld, 0);
    }
    ok = __syncthreads_and(ok) != 0;   // one decision for the whole CTA
    // FP8: scale exponent of each block of rows_per_scale rows (the tile holds
    // whole blocks), from the largest magnitude any of its rows reads
    if (PREC == RX_FIR_FP8) {
        float m = 0.f;
        if (tid < rows) {
            const float2 *x = stage + shift + 2 * kRowSyms * tid;
            for (int s = 0; s < ns; s++) m = fmaxf(m, fmaxf(fabsf(x[s].x), fabsf(x[s].y)));
        }
        reinterpret_cast<float *>(s_exp)[tid] = m;
        __syncthreads();
        if (tid < kTileRows / rows_per_scale) {
            float bm = 0.f;
            for (int r = tid * rows_per_scale; r < (tid + 1) * rows_per_scale; r++)
                bm = fmaxf(bm, reinterpret_cast<float *>(s_exp)[r]);
            m = bm;
        }
        __syncthreads();
        if (tid < kTileRows / rows_per_scale) s_exp[tid] = fp8_exp(m);
        __syncthreads();
    }
    // A: row r, K index k -> staged float 2 (shift + 32 r) + k for k < 2 ns, else 0
    for (int u = tid; u < kTileRows * PLANES; u += kThreads) {
        int r = u % kTileRows, pl = u / kTileRows;
        float v[16];
        const float *src = reinterpret_cast<const float *>(stage + shift + 2 * kRowSyms * r) + pl * EPP;
#pragma unroll
        for (int t = 0; t < EPP; t++) v[t] = (r < rows && pl * EPP + t < 2 * ns) ? src[t] : 0.f;
        float sAv = PREC == RX_FIR_FP8 ? ldexpf(1.f, s_exp[r / rows_per_scale]) : 1.f;
        *reinterpret_cast<uint4 *>(sA + pl * PLANE_A + r * 16) = pack16<PREC>(v, sAv);
    }
    fence_async_smem();
    __syncthreads();

    if (tid == 0 && ok) {
        tc_fence_after();
        const uint32_t idesc = umma_idesc(Fmt<PREC>::code, kTileRows, kN);
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
        for (int q = 0; q < NMMA; q++) {
            uint64_t ad = umma_sdesc(a0 + q * 2 * PLANE_A, PLANE_A, 128);
            uint64_t bd = umma_sdesc(b0 + q * 2 * PLANE_B, PLANE_B, 128);
            if (PREC == RX_FIR_FP8) umma_f8(tmem, ad, bd, idesc, q > 0);
            else umma_f16(tmem, ad, bd, idesc, q > 0);
        }
        umma_commit(bar_mma);
    }
    if (ok) {
        bool done = mbar_wait(bar_mma, 0);
        if (!done) {
            atomicExch(err, (int)RX_ETIMEOUT);
            mbar_wait(bar_mma, 0);
        }
        ok = done;
    }
    ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
    if (ok) {
        // epilogue: warp w owns accumulator lanes 32w..32w+31 (= rows)
        uint32_t acc[32];
        tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), acc);
        int r = 32 * warp + lane;
        if (r < rows) {
            float inv = 1.f;
            if (PREC == RX_FIR_FP8) inv = ldexpf(1.f, -(eB + s_exp[r / rows_per_scale]));
            float4 *dst = reinterpret_cast<float4 *>(z + (long long)(r0 + r) * kRowSyms);
#pragma unroll
            for (int q = 0; q < kRowSyms / 2; q++)
                dst[q] = make_float4(__uint_as_float(acc[4 * q]) * inv, __uint_as_float(acc[4 * q + 1]) * inv,
                                     __uint_as_float(acc[4 * q + 2]) * inv, __uint_as_float(acc[4 * q + 3]) * inv);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

cudaError_t launch_fir_tc(int prec, const float2 *Y, long long ybase, long long k_lo, long long nsym,
                          const float2 *taps, int ntaps, int scale_block, float2 *z, int *err, cudaStream_t st)
{
    if (nsym <= 0) return cudaSuccess;
    if (nsym % kRowSyms || ntaps < 1 || ntaps > 31 || !(ntaps & 1) || scale_block % kRowSyms ||
        (kTileRows * kRowSyms) % scale_block)
        return cudaErrorInvalidValue;
    int nrows = (int)(nsym / kRowSyms);
    int rps = scale_block / kRowSyms;
    unsigned grid = (unsigned)((nrows + kTileRows - 1) / kTileRows);
#define RX_FIR_LAUNCH(P)                                                                                     \
    do {                                                                                                     \
        cudaFuncSetAttribute(k_fir_tc<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);               \
        k_fir_tc<P><<<grid, kThreads, kSmem, st>>>(Y, ybase, k_lo, nrows, taps, ntaps, rps, z, err);         \
    } while (0)
    switch (prec) {
    case RX_FIR_BF16: RX_FIR_LAUNCH(RX_FIR_BF16); break;
    case RX_FIR_FP16: RX_FIR_LAUNCH(RX_FIR_FP16); break;
    case RX_FIR_FP8: RX_FIR_LAUNCH(RX_FIR_FP8); break;
    default: return cudaErrorInvalidValue;
    }
#undef RX_FIR_LAUNCH
    return cudaGetLastError();
}

}  // namespace rxk
