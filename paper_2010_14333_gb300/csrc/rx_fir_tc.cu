// Block-Toeplitz FIR on the fifth-generation tensor cores (tcgen05).
//
// The equaliser's filter z_k = sum_i conj(w_i) y[2k + TH - i] with taps that are
// fixed for a whole call (the frozen form) is one dense contraction: rows of 16
// consecutive symbols, each row a K = 2 (30 + NT) real slice (padded to 128) of
// the 2-sps sequence as stored (complex interleaved; consecutive rows overlap,
// a Hankel matrix), times a K x 32 real Toeplitz matrix of the taps (complex
// split to real: re / im output of each symbol).  Tiles of 128 rows (2048
// symbols) run through M = 128, N = 32 tcgen05.mma in BF16, FP16 or FP8-E4M3
// with FP32 accumulation in tensor memory.  Persistent CTAs (two per SM), per
// tile:
//   - a bulk copy (cp.async.bulk) stages the next tile's 4.1 k complex FP32
//     inputs while this tile is processed (two stage buffers, one mbarrier each);
//   - the threads convert the staged inputs into the K-major no-swizzle operand
//     layout (core matrices of 8 rows x 16 bytes), lanes spread over 8 rows x 4
//     K-columns with a rotated read order so that neither the shared-memory reads
//     nor the 16-byte stores conflict; FP8 first takes a power-of-two scale per
//     block of rows_per_scale rows from the block's largest input;
//   - one thread issues the MMAs and commits them to an mbarrier;
//   - each warp reads its 32 accumulator lanes (tcgen05.ld 32x32b), rescales,
//     transposes through shared memory and stores 512 contiguous bytes per
//     instruction.
// The taps' Toeplitz operand is built once per CTA.  Every wait is bounded: on
// time-out the kernel records RX_ETIMEOUT, waits (bounded) for its own copies and
// MMAs, frees its tensor memory and returns.
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
constexpr int kThreads = 256;            // 8 warps: (row quarter, K / column half)
constexpr int kStage = 2 * kRowSyms * kTileRows + 64;   // staged complex inputs per tile
constexpr int kOutPitch = kN + 4;                  // floats per row of the output transpose
constexpr uint32_t kTmemCols = 32;
// dynamic shared memory: A | B | stage[2] | barriers and scratch
constexpr int kOffA = 0;
constexpr int kOffB = kOffA + kTileRows * kKP * 2;   // 32 KB (16-bit A; FP8 uses half)
constexpr int kOffStage = kOffB + kN * kKP * 2;      // + 8 KB
constexpr int kStageBytes = kStage * 8;
constexpr int kOffMisc = kOffStage + 2 * kStageBytes;
// misc: 3 mbarriers + TMEM slot (64 B) | per-row maxima (128 floats) | scale exponents (128 ints)
constexpr int kOffRmax = kOffMisc + 64;                 // float [2 halves][128 rows]
constexpr int kOffExp = kOffRmax + 2 * kTileRows * 4;
constexpr int kSmem = kOffExp + kTileRows * 4;
static_assert(kTileRows * kOutPitch * 4 <= kStageBytes, "output transpose fits a stage buffer");
static_assert(kSmem <= 113 * 1024, "two CTAs per SM");

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
__global__ void __launch_bounds__(kThreads, 2)
    k_fir_tc(const float2 *__restrict__ Y, long long ybase, long long k_lo, int nrows,
             const float2 *__restrict__ taps, int ntaps, int rows_per_scale, float2 *__restrict__ z, int *err)
{
    constexpr int ES = Fmt<PREC>::esize;
    constexpr int EPP = 16 / ES;                    // K elements per 16-byte core row
    constexpr int PLANES = kKP / EPP;               // K core-matrix columns (16 or 8)
    constexpr int PLANE_A = kTileRows * 16, PLANE_B = kN * 16;
    constexpr int NMMA = PLANES / 2;                // each MMA consumes two K core matrices
    constexpr int F2 = EPP / 2;                     // float2 reads per (row, plane)
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sA = sm + kOffA, *sB = sm + kOffB;
    uint64_t *bar_ld = reinterpret_cast<uint64_t *>(sm + kOffMisc);   // [2]
    uint64_t *bar_mma = bar_ld + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_ld + 3);
    float *s_rmax = reinterpret_cast<float *>(sm + kOffRmax);          // [2][128]
    int *s_exp = reinterpret_cast<int *>(sm + kOffExp);                // [<= 128]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, quarter = warp & 3, half = warp >> 2;
    const int th = (ntaps - 1) / 2;
    const int ns = 2 * kRowSyms - 2 + ntaps;       // complex inputs per row
    const int ntiles = (nrows + kTileRows - 1) / kTileRows;

    // staged range of tile t: from an even element offset, so the copy starts on 16 bytes
    auto tile_src = [&](int t, long long &es, int &shift, int &nst) {
        int r0 = t * kTileRows, rows = min(kTileRows, nrows - r0);
        long long e0 = 2 * (k_lo + (long long)r0 * kRowSyms) - th - ybase;
        es = e0 & ~1LL;
        shift = (int)(e0 - es);
        nst = ((shift + 2 * kRowSyms * (rows - 1) + ns) + 1) & ~1;
    };
    auto issue = [&](int t, int buf) {
        long long es;
        int shift, nst;
        tile_src(t, es, shift, nst);
        fence_async_smem();   // earlier generic writes to this buffer precede the copy
        mbar_expect_tx(bar_ld + buf, (unsigned)(nst * 8));
        bulk_g2s(sm + kOffStage + buf * kStageBytes, Y + es, (unsigned)(nst * 8), bar_ld + buf);
    };
    if (tid == 0) {
        mbar_init(bar_ld, 1);
        mbar_init(bar_ld + 1, 1);
        mbar_init(bar_mma, 1);
        if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
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
    const uint32_t idesc = umma_idesc(Fmt<PREC>::code, kTileRows, kN);

    // lane -> (row r_lo, K column p_lo) of an 8 x 4 group; a warp's groups cover
    // the 32 rows of its lane quarter and half of the K columns
    const int r_lo = lane & 7, p_lo = lane >> 3, rot = r_lo % F2;
    bool ok = true;
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {
        const int buf = it & 1;
        const int r0 = t * kTileRows, rows = min(kTileRows, nrows - r0);
        long long es;
        int shift, nst;
        tile_src(t, es, shift, nst);
        if (tid == 0 && t + (int)gridDim.x < ntiles) issue(t + gridDim.x, buf ^ 1);   // prefetch
        bool got = mbar_wait(bar_ld + buf, (unsigned)((it >> 1) & 1));
        if (!got) {
            atomicExch(err, (int)RX_ETIMEOUT);
            mbar_wait(bar_ld + buf, (unsigned)((it >> 1) & 1));
        }
        ok = __syncthreads_and(got) != 0;
        if (!ok) break;
        const float *stf = reinterpret_cast<const float *>(sm + kOffStage + buf * kStageBytes) + 2 * shift;

        // (row, K column) -> the 16 bytes of K elements it holds, read in a rotated
        // order; returns the EPP floats in natural order
        auto load_unit = [&](int r, int pl, float (&v)[16]) {
            const float *base = stf + 4 * kRowSyms * r + pl * EPP;   // rows start 2 kRowSyms complex apart
            float2 tmp[F2];
#pragma unroll
            for (int q = 0; q < F2; q++) {
                int qq = (q + rot) % F2;
                tmp[q] = *reinterpret_cast<const float2 *>(base + 2 * qq);
            }
#pragma unroll
            for (int q = 0; q < F2; q++) {
                // undo the rotation: element qq came in slot (qq - rot) mod F2
                float2 e = tmp[0];
#pragma unroll
                for (int u = 1; u < F2; u++)
                    if (((q - rot + F2) % F2) == u) e = tmp[u];
                v[2 * q] = e.x;
                v[2 * q + 1] = e.y;
            }
#pragma unroll
            for (int u = 0; u < EPP; u++)
                if (r >= rows || pl * EPP + u >= 2 * ns) v[u] = 0.f;
        };

        if (PREC == RX_FIR_FP8) {
            // per-row largest input magnitude, then per scale block
#pragma unroll 1
            for (int rh = 0; rh < 4; rh++) {
                int r = 32 * quarter + 8 * rh + r_lo;
                float m = 0.f;
#pragma unroll 1
                for (int ph = half * (PLANES / 8); ph < (half + 1) * (PLANES / 8); ph++) {
                    float v[16];
                    load_unit(r, 4 * ph + p_lo, v);
#pragma unroll
                    for (int u = 0; u < EPP; u++) m = fmaxf(m, fabsf(v[u]));
                }
                m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 8));
                m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));
                if (p_lo == 0) s_rmax[half * kTileRows + r] = m;
            }
            __syncthreads();
            if (tid < kTileRows / rows_per_scale) {
                float bm = 0.f;
                for (int r = tid * rows_per_scale; r < (tid + 1) * rows_per_scale; r++)
                    bm = fmaxf(bm, fmaxf(s_rmax[r], s_rmax[kTileRows + r]));
                s_exp[tid] = fp8_exp(bm);
            }
            __syncthreads();
        }
        // A: row r, K index k -> staged float 2 (shift + 32 r) + k for k < 2 ns, else 0
#pragma unroll 1
        for (int rh = 0; rh < 4; rh++) {
            int r = 32 * quarter + 8 * rh + r_lo;
            float sAv = PREC == RX_FIR_FP8 ? ldexpf(1.f, s_exp[r / rows_per_scale]) : 1.f;
#pragma unroll 2
            for (int ph = half * (PLANES / 8); ph < (half + 1) * (PLANES / 8); ph++) {
                int pl = 4 * ph + p_lo;
                float v[16];
                load_unit(r, pl, v);
                *reinterpret_cast<uint4 *>(sA + pl * PLANE_A + r * 16) = pack16<PREC>(v, sAv);
            }
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
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
        bool done = mbar_wait(bar_mma, (unsigned)(it & 1));
        if (!done) {
            atomicExch(err, (int)RX_ETIMEOUT);
            mbar_wait(bar_mma, (unsigned)(it & 1));
        }
        ok = __syncthreads_and(done) != 0;
        if (!ok) break;
        tc_fence_after();
        // epilogue: warp (quarter, half) owns accumulator lanes 32 quarter .. + 31 (rows)
        // and columns 16 half .. + 15; rows go through the consumed stage buffer to
        // leave as contiguous 512-byte stores
        {
            uint32_t acc[16];
            tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + 16 * half, acc);
            const int r = 32 * quarter + lane;
            float inv = 1.f;
            if (PREC == RX_FIR_FP8) inv = ldexpf(1.f, -(eB + s_exp[r / rows_per_scale]));
            float *ot = reinterpret_cast<float *>(sm + kOffStage + buf * kStageBytes);
#pragma unroll
            for (int q = 0; q < 4; q++)
                *reinterpret_cast<float4 *>(ot + r * kOutPitch + 16 * half + 4 * q) =
                    make_float4(__uint_as_float(acc[4 * q]) * inv, __uint_as_float(acc[4 * q + 1]) * inv,
                                __uint_as_float(acc[4 * q + 2]) * inv, __uint_as_float(acc[4 * q + 3]) * inv);
            __syncthreads();
            float4 *zt = reinterpret_cast<float4 *>(z + (long long)r0 * kRowSyms);
            for (int i = tid; i < kTileRows * 8; i += kThreads) {
                int rr = i >> 3, ch = i & 7;
                if (rr < rows) zt[rr * 8 + ch] = *reinterpret_cast<const float4 *>(ot + rr * kOutPitch + 4 * ch);
            }
        }
        tc_fence_before();
        __syncthreads();   // A, the accumulator and this stage buffer are free again
    }
    if (!ok && tid == 0) {
        // a prefetch may still be in flight: wait for it (bounded) before leaving
        mbar_wait(bar_ld + ((it + 1) & 1), (unsigned)(((it + 1) >> 1) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}


// ---------------------------------------------------------------------------
// 16-bit forms (BF16, FP16): each input sample is converted once.  Block row q of
// a tile holds the 32 complex samples that start at stream sample
// 2 (k_lo + 16 (r0 + q)) - 16, i.e. 64 K elements in 8 core-matrix columns whose
// rows lie 16 bytes apart across 8-row groups (SBO = 128).  Output row r (symbols
// k = k_lo + 16 (r0 + r) + j, j < 16) needs samples 2k - TH .. 2k + TH with TH <= 15,
// all inside block rows r and r + 1: the tile is X[r] B0 + X[r + 1] B1, two sets
// of four K = 16 MMAs over the same planes, the second with its descriptors
// shifted by one row (16 bytes).  Persistent CTAs, two per SM: the next tile's
// samples are loaded into registers while this tile's MMAs and stores run (a
// launch of one CTA per tile spent its first 4 us bringing 512 CTAs up).
constexpr int kT2Rows = kTileRows + 8;            // block rows a plane holds (129 used)
constexpr int kT2Plane = kT2Rows * 16 + 16;       // plane pitch: + 16 bytes skews the planes by 4 banks
constexpr int kT2Planes = 2 * kRowSyms * 2 / 8;   // 64 K elements of a block row, 8 per core row
constexpr int kT2BPlane = kN * 16;                // one K core-matrix column of B (32 rows)
constexpr int kT2OffB = kT2Planes * kT2Plane;
constexpr int kT2OffW = kT2OffB + 2 * kT2Planes * kT2BPlane;   // the taps (32 complex)
constexpr int kT2OffBar = kT2OffW + 32 * 8;
constexpr int kT2Smem = kT2OffBar + 16;
constexpr int kT2Threads = 256;
constexpr int kT2Samples = (kTileRows + 1) * 2 * kRowSyms;   // complex samples a tile converts
constexpr int kT2Iter = (kT2Samples + kT2Threads - 1) / kT2Threads;
static_assert(kT2Plane % 16 == 0 && kT2OffB % 16 == 0 && kT2OffBar % 8 == 0, "16-byte aligned operands");
static_assert((kT2Plane / 4) % 32 == 4, "planes four banks apart: a warp's 32 samples store conflict-free");

template <int PREC>
__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    if (PREC == RX_FIR_BF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}

template <int PREC>
__global__ void __launch_bounds__(kT2Threads, 2)
    k_fir_tc2(const float2 *__restrict__ Y, long long ybase, long long k_lo, int nrows,
              const float2 *__restrict__ taps, int ntaps, float2 *__restrict__ z, int *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sA = sm, *sB = sm + kT2OffB;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kT2OffBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    float2 *s_w = reinterpret_cast<float2 *>(sm + kT2OffW);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, quarter = warp & 3, half = warp >> 2;
    const int th = (ntaps - 1) / 2;
    const int ntiles = (nrows + kTileRows - 1) / kTileRows;
    // a tile's samples into registers: sample j of tile t is stream sample
    // 2 (k_lo + 16 r0) - 16 + j; zero outside the samples its symbols use, so that
    // nothing outside the caller's range is read
    float2 v[kT2Iter];
    auto load_tile = [&](int t) {
        const int r0 = t * kTileRows, rows = min(kTileRows, nrows - r0);
        const long long n0 = 2 * (k_lo + (long long)r0 * kRowSyms) - 16;
        const int jlo = 16 - th, jhi = 2 * (rows * kRowSyms - 1) + th + 16;
        const float2 *Yb = Y + (n0 - ybase);
#pragma unroll
        for (int i = 0; i < kT2Iter; i++) {
            const int j = tid + i * kT2Threads;
            v[i] = (j >= jlo && j <= jhi && j < kT2Samples) ? __ldg(Yb + j) : make_float2(0.f, 0.f);
        }
    };
    int t = blockIdx.x;
    if (tid < 32) s_w[tid] = tid < ntaps ? __ldg(taps + tid) : make_float2(0.f, 0.f);
    if (t < ntiles) load_tile(t);
    if (tid == 0) mbar_init(bar, 1);
    if (warp == 0) tmem_alloc(tslot, kTmemCols);
    __syncthreads();   // the taps in shared memory
    // B: rows n = 2 j + c (c: re / im output of symbol j), K index k = 64 h + 2 s + d
    // (block row r + h, sample s, d: re / im); sample 32 h + s of the pair is stream
    // sample 2 k_row - 16 + 32 h + s, so tap i = 2 j + TH + 16 - (32 h + s)
    for (int u = tid; u < kN * 2 * kT2Planes; u += kT2Threads) {
        const int n = u % kN, pl = u / kN;
        const int j = n >> 1, c = n & 1;
        float vb[16];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int k = 8 * pl + q, hb = k >> 6, sp = (k & 63) >> 1, d = k & 1;
            const int i = 2 * j + th + 16 - (32 * hb + sp);
            float val = 0.f;
            if (i >= 0 && i < ntaps) {
                const float2 w = s_w[i];
                // conj(w) y: re = a yr + b yi, im = a yi - b yr
                val = c == 0 ? (d == 0 ? w.x : w.y) : (d == 0 ? -w.y : w.x);
            }
            vb[q] = val;
        }
        *reinterpret_cast<uint4 *>(sB + pl * kT2BPlane + n * 16) = pack16<PREC>(vb, 1.f);
    }
    const uint32_t idesc = umma_idesc(Fmt<PREC>::code, kTileRows, kN);
    bool ok = true;
    for (int it = 0; t < ntiles; t += gridDim.x, it++) {
        const int r0 = t * kTileRows, rows = min(kTileRows, nrows - r0);
        // A: sample j of the tile -> block row j / 32, K elements 2 (j % 32) and + 1
#pragma unroll
        for (int i = 0; i < kT2Iter; i++) {
            const int j = tid + i * kT2Threads;
            if (j < kT2Samples) {
                const int q = j >> 5, s = j & 31;
                *reinterpret_cast<uint32_t *>(sA + (s >> 2) * kT2Plane + q * 16 + (s & 3) * 4) =
                    pack2<PREC>(v[i].x, v[i].y);
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        const uint32_t tmem = *tslot;
        // the next tile's loads are in flight while this tile's MMAs and stores run
        if (t + (int)gridDim.x < ntiles) load_tile(t + gridDim.x);
        if (tid == 0) {
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int q = 0; q < kT2Planes; q++) {
                const uint32_t shift = q < kT2Planes / 2 ? 0u : 16u;   // block row r, then r + 1
                const uint64_t ad = umma_sdesc(a0 + shift + (q % (kT2Planes / 2)) * 2 * kT2Plane, kT2Plane, 128);
                const uint64_t bd = umma_sdesc(b0 + q * 2 * kT2BPlane, kT2BPlane, 128);
                umma_f16(tmem, ad, bd, idesc, q > 0);
            }
            umma_commit(bar);
        }
        bool done = mbar_wait(bar, (unsigned)(it & 1));
        if (!done) {
            atomicExch(err, (int)RX_ETIMEOUT);
            mbar_wait(bar, (unsigned)(it & 1));
        }
        ok = __syncthreads_and(done) != 0;
        tc_fence_after();
        if (!ok) break;
        // warp (quarter, half): accumulator lanes (rows) 32 quarter .. + 31, columns
        // 16 half .. + 15 = symbols 8 half .. + 7 of the row, stored as four 16-byte pieces
        uint32_t acc[16];
        tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + 16 * half, acc);
        const int r = 32 * quarter + lane;
        if (r < rows) {
            float4 *zr = reinterpret_cast<float4 *>(z + ((long long)(r0 + r) * kRowSyms + 8 * half));
#pragma unroll
            for (int q = 0; q < 4; q++)
                zr[q] = make_float4(__uint_as_float(acc[4 * q]), __uint_as_float(acc[4 * q + 1]),
                                    __uint_as_float(acc[4 * q + 2]), __uint_as_float(acc[4 * q + 3]));
        }
        tc_fence_before();
        __syncthreads();   // A and the accumulator are free again
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(*tslot, kTmemCols);
}

}  // namespace

cudaError_t prepare_fir_tc(int prec)
{
    switch (prec) {
    case RX_FIR_BF16:
    case RX_FIR_FP16: return cudaSuccess;   // the 16-bit kernel's shared memory is under the default limit
    case RX_FIR_FP8: return cudaFuncSetAttribute(k_fir_tc<RX_FIR_FP8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fir_tc(int prec, const float2 *Y, long long ybase, long long k_lo, long long nsym,
                          const float2 *taps, int ntaps, int scale_block, float2 *z, int *err, int nsm,
                          cudaStream_t st)
{
    if (nsym <= 0) return cudaSuccess;
    if (nsym % kRowSyms || ntaps < 1 || ntaps > 31 || !(ntaps & 1) || scale_block % kRowSyms ||
        (kTileRows * kRowSyms) % scale_block)
        return cudaErrorInvalidValue;
    int nrows = (int)(nsym / kRowSyms);
    int rps = scale_block / kRowSyms;
    int ntiles = (nrows + kTileRows - 1) / kTileRows;
    if (prec == RX_FIR_BF16 || prec == RX_FIR_FP16) {
        const unsigned g2 = (unsigned)min(ntiles, 2 * nsm);   // two persistent CTAs per SM
        if (prec == RX_FIR_BF16)
            k_fir_tc2<RX_FIR_BF16><<<g2, kT2Threads, kT2Smem, st>>>(Y, ybase, k_lo, nrows, taps, ntaps, z, err);
        else
            k_fir_tc2<RX_FIR_FP16><<<g2, kT2Threads, kT2Smem, st>>>(Y, ybase, k_lo, nrows, taps, ntaps, z, err);
        return cudaGetLastError();
    }
    unsigned grid = (unsigned)min(ntiles, 2 * nsm);   // two persistent CTAs per SM
#define RX_FIR_LAUNCH(P) k_fir_tc<P><<<grid, kThreads, kSmem, st>>>(Y, ybase, k_lo, nrows, taps, ntaps, rps, z, err)
    if (prec != RX_FIR_FP8) return cudaErrorInvalidValue;
    RX_FIR_LAUNCH(RX_FIR_FP8);
#undef RX_FIR_LAUNCH
    return cudaGetLastError();
}

}  // namespace rxk
