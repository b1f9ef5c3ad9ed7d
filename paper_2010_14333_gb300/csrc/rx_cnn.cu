// Learned equaliser: a 1-D CNN over the 2-sps matched-filter output, trained on
// the GPU by its own forward and backward kernels (BF16 operands on the tensor
// cores for the forward convolutions, FP32 accumulation, FP32 master weights and
// Adam).
//
// Network (the configured workload's learned equaliser): input y as two channels
// (real, imaginary); three valid convolutions of 32 channels, kernel 9, each
// followed by GELU (exact erf form); at every symbol position an MLP
// 32 -> 64 (GELU) -> 2 gives the soft symbol in unit-power units.  A segment of
// S = 64 symbols starting at symbol k0 reads y[2 k0 - 12, 2 k0 + 140).
// Parameter vector: W1[32][9][2] b1[32] W2[32][9][32] b2[32] W3[32][9][32] b3[32]
//                   M1[64][32] c1[64] M2[2][64] c2[2].
// Activations are channel-last, so the im2col row of output position p of a
// 32-channel layer is the contiguous slice act[32 p, 32 p + 288): the
// convolution is a plain GEMM A[p][k] = act[32 p + k], k = 9 x 32, against
// W[o][k], computed with mma.sync m16n8k16 (BF16 in, FP32 accumulate).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "rx_async.cuh"
#include "rx_common.cuh"
#include "rx_internal.cuh"

namespace rxk {

constexpr int CC = 32, CK = 9, CH = 64, CS = 64;          // channels, kernel, hidden, symbols per segment
constexpr int L0 = 2 * CS + 24, L1 = L0 - 8, L2 = L1 - 8, L3 = L2 - 8;
constexpr int KW = CK * CC;                               // 288
constexpr int OW1 = 0, OB1 = OW1 + CC * CK * 2, OW2 = OB1 + CC, OB2 = OW2 + CC * KW, OW3 = OB2 + CC,
              OB3 = OW3 + CC * KW, OM1 = OB3 + CC, OC1 = OM1 + CH * CC, OM2 = OC1 + CH, OC2 = OM2 + 2 * CH,
              NPRM = OC2 + 2;
constexpr int kCnnThreads = 128;

__device__ __forceinline__ float gelu_f(float u) { return 0.5f * u * (1.0f + erff(u * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_df(float u)
{
    return 0.5f * (1.0f + erff(u * 0.70710678118654752f)) + u * 0.3989422804014327f * __expf(-0.5f * u * u);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// saved forward state of one segment (training)
struct CnnSave {
    float *u1, *u2, *u3;          // pre-activations, [seg][L][32]
    __nv_bfloat16 *h1, *h2, *h3;  // activations, [seg][L][32]
    float *v;                     // MLP pre-activation, [seg][S][64]
    float *out;                   // outputs, [seg][S][2]
};

// 32-channel valid convolution layer on the tensor cores:
// dst[p][o] = GELU(b[o] + sum_k src[32 p + k] W[o][k]) for p < Lout; src has at
// least 16 * ceil(Lout / 16) + 8 rows (extra rows zero).
template <int LOUT>
__device__ __forceinline__ void conv32_mma(const __nv_bfloat16 *src, const __nv_bfloat16 *W, const float *b,
                                           __nv_bfloat16 *dst, float *u_save, int warp, int lane)
{
    constexpr int TILES = (LOUT + 15) / 16;
    const int g = lane >> 2, tq = lane & 3;
    for (int tile = warp; tile < TILES; tile += kCnnThreads / 32) {
        const int r0 = 16 * tile;
        float acc[4][4];
#pragma unroll
        for (int n = 0; n < 4; n++)
#pragma unroll
            for (int i = 0; i < 4; i++) acc[n][i] = 0.f;
#pragma unroll 2
        for (int k0 = 0; k0 < KW; k0 += 16) {
            uint32_t a[4];
            const __nv_bfloat16 *ar = src + 32 * (r0 + g) + k0 + 2 * tq;
            a[0] = *reinterpret_cast<const uint32_t *>(ar);
            a[1] = *reinterpret_cast<const uint32_t *>(ar + 32 * 8);
            a[2] = *reinterpret_cast<const uint32_t *>(ar + 8);
            a[3] = *reinterpret_cast<const uint32_t *>(ar + 32 * 8 + 8);
#pragma unroll
            for (int n = 0; n < 4; n++) {
                const __nv_bfloat16 *br = W + KW * (8 * n + g) + k0 + 2 * tq;
                mma_bf16(acc[n], a, *reinterpret_cast<const uint32_t *>(br),
                         *reinterpret_cast<const uint32_t *>(br + 8));
            }
        }
#pragma unroll
        for (int n = 0; n < 4; n++)
#pragma unroll
            for (int i = 0; i < 4; i++) {
                int r = r0 + g + 8 * (i >> 1), o = 8 * n + 2 * tq + (i & 1);
                if (r < LOUT) {
                    float u = acc[n][i] + b[o];
                    dst[32 * r + o] = __float2bfloat16(gelu_f(u));
                    if (u_save) u_save[32 * r + o] = u;
                }
            }
    }
}

// shared-memory layout of the forward kernel (bytes)
struct FwdSmem {
    static constexpr int X = 0;                                     // float [L0][2]
    static constexpr int W1 = X + L0 * 2 * 4;                       // float [32][18]
    static constexpr int B = W1 + CC * 18 * 4;                      // float b1, b2, b3 [96]
    static constexpr int M1 = B + 3 * CC * 4;                       // float [64][32]
    static constexpr int C1 = M1 + CH * CC * 4;                     // float [64]
    static constexpr int M2 = C1 + CH * 4;                          // float [2][64] + c2 [2]
    static constexpr int WB2 = ((M2 + (2 * CH + 2) * 4) + 15) & ~15; // bf16 [32][288]
    static constexpr int WB3 = WB2 + CC * KW * 2;
    static constexpr int H1 = WB3 + CC * KW * 2;                    // bf16 [L1 + 16][32]
    static constexpr int H2 = H1 + (L1 + 16) * CC * 2;              // bf16 [L2 + 16][32]
    static constexpr int H3 = H2 + (L2 + 16) * CC * 2;              // bf16 [L3][32]
    static constexpr int OUT = H3 + L3 * CC * 2;                    // float [S][2]
    static constexpr int TOTAL = OUT + CS * 2 * 4;
};

// Forward pass of nseg segments, one CTA each.  y: complex 2-sps input; seg_start[s]:
// index in y of the segment's first input sample (2 k0 - 12).  Writes out[s][j][2]
// and, when sv.u1 is set, the activations for the backward pass.  In receiver mode
// (dec non-null) it decides the symbols instead and scores them (window records).
__global__ void __launch_bounds__(kCnnThreads)
    k_cnn_fwd(const float *__restrict__ prm, const __nv_bfloat16 *__restrict__ prm_bf, const float2 *__restrict__ y,
              const long long *__restrict__ seg_start, long long seg_base, long long seg_step, float *__restrict__ out,
              CnnSave sv, uint8_t *__restrict__ dec, uint8_t *__restrict__ winb, uint4 *__restrict__ winrec,
              const uint32_t *__restrict__ prbs_bits, long long k_first, float scale, int mq)
{
    extern __shared__ __align__(16) unsigned char sm[];
    float *xs = reinterpret_cast<float *>(sm + FwdSmem::X);
    float *w1 = reinterpret_cast<float *>(sm + FwdSmem::W1);
    float *bb = reinterpret_cast<float *>(sm + FwdSmem::B);
    float *m1 = reinterpret_cast<float *>(sm + FwdSmem::M1);
    float *c1 = reinterpret_cast<float *>(sm + FwdSmem::C1);
    float *m2 = reinterpret_cast<float *>(sm + FwdSmem::M2);
    __nv_bfloat16 *wb2 = reinterpret_cast<__nv_bfloat16 *>(sm + FwdSmem::WB2);
    __nv_bfloat16 *wb3 = reinterpret_cast<__nv_bfloat16 *>(sm + FwdSmem::WB3);
    __nv_bfloat16 *h1 = reinterpret_cast<__nv_bfloat16 *>(sm + FwdSmem::H1);
    __nv_bfloat16 *h2 = reinterpret_cast<__nv_bfloat16 *>(sm + FwdSmem::H2);
    __nv_bfloat16 *h3 = reinterpret_cast<__nv_bfloat16 *>(sm + FwdSmem::H3);
    float *os = reinterpret_cast<float *>(sm + FwdSmem::OUT);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s = blockIdx.x;
    const long long st = seg_start ? seg_start[s] : seg_base + seg_step * s;
    // stage inputs and parameters
    for (int i = tid; i < L0; i += kCnnThreads) {
        float2 v = y[st + i];
        xs[2 * i] = v.x;
        xs[2 * i + 1] = v.y;
    }
    for (int i = tid; i < CC * 18; i += kCnnThreads) w1[i] = prm[OW1 + i];
    for (int i = tid; i < CC; i += kCnnThreads) {
        bb[i] = prm[OB1 + i];
        bb[CC + i] = prm[OB2 + i];
        bb[2 * CC + i] = prm[OB3 + i];
    }
    for (int i = tid; i < CH * CC; i += kCnnThreads) m1[i] = prm[OM1 + i];
    for (int i = tid; i < CH; i += kCnnThreads) c1[i] = prm[OC1 + i];
    for (int i = tid; i < 2 * CH + 2; i += kCnnThreads) m2[i] = prm[OM2 + i];
    for (int i = tid; i < CC * KW / 8; i += kCnnThreads) {
        reinterpret_cast<uint4 *>(wb2)[i] = reinterpret_cast<const uint4 *>(prm_bf + OW2)[i];
        reinterpret_cast<uint4 *>(wb3)[i] = reinterpret_cast<const uint4 *>(prm_bf + OW3)[i];
    }
    // zero the padding rows read by the last (partial) row tiles
    for (int i = tid; i < 16 * CC; i += kCnnThreads) {
        h1[L1 * CC + i] = __float2bfloat16(0.f);
        h2[L2 * CC + i] = __float2bfloat16(0.f);
    }
    __syncthreads();
    // layer 1 (2 input channels, K = 18) on the CUDA cores
    float *u1s = sv.u1 ? sv.u1 + (size_t)s * L1 * CC : nullptr;
    for (int i = tid; i < L1 * CC; i += kCnnThreads) {
        int p = i >> 5, o = i & 31;
        float a = bb[o];
#pragma unroll
        for (int k = 0; k < 18; k++) a = fmaf(w1[o * 18 + k], xs[2 * p + k], a);
        h1[i] = __float2bfloat16(gelu_f(a));
        if (u1s) u1s[i] = a;
    }
    __syncthreads();
    conv32_mma<L2>(h1, wb2, bb + CC, h2, sv.u2 ? sv.u2 + (size_t)s * L2 * CC : nullptr, warp, lane);
    __syncthreads();
    conv32_mma<L3>(h2, wb3, bb + 2 * CC, h3, sv.u3 ? sv.u3 + (size_t)s * L3 * CC : nullptr, warp, lane);
    __syncthreads();
    if (sv.h1) {
        for (int i = tid; i < L1 * CC / 8; i += kCnnThreads)
            reinterpret_cast<uint4 *>(sv.h1 + (size_t)s * L1 * CC)[i] = reinterpret_cast<const uint4 *>(h1)[i];
        for (int i = tid; i < L2 * CC / 8; i += kCnnThreads)
            reinterpret_cast<uint4 *>(sv.h2 + (size_t)s * L2 * CC)[i] = reinterpret_cast<const uint4 *>(h2)[i];
        for (int i = tid; i < L3 * CC / 8; i += kCnnThreads)
            reinterpret_cast<uint4 *>(sv.h3 + (size_t)s * L3 * CC)[i] = reinterpret_cast<const uint4 *>(h3)[i];
    }
    // MLP head at the symbol positions: two threads per symbol, 32 hidden units each
    {
        int j = tid >> 1, half = tid & 1;
        float hv[CC];
#pragma unroll
        for (int c = 0; c < CC; c++) hv[c] = __bfloat162float(h3[(2 * j) * CC + c]);
        float o0 = 0.f, o1 = 0.f;
        for (int mm = 0; mm < CH / 2; mm++) {
            int m = half * (CH / 2) + mm;
            float a = c1[m];
#pragma unroll
            for (int c = 0; c < CC; c++) a = fmaf(m1[m * CC + c], hv[c], a);
            if (sv.v) sv.v[((size_t)s * CS + j) * CH + m] = a;
            float z = gelu_f(a);
            o0 = fmaf(m2[m], z, o0);
            o1 = fmaf(m2[CH + m], z, o1);
        }
        o0 += __shfl_xor_sync(0xffffffffu, o0, 1);
        o1 += __shfl_xor_sync(0xffffffffu, o1, 1);
        if (!half) {
            o0 += m2[2 * CH];
            o1 += m2[2 * CH + 1];
            os[2 * j] = o0;
            os[2 * j + 1] = o1;
            if (out) {
                out[((size_t)s * CS + j) * 2] = o0;
                out[((size_t)s * CS + j) * 2 + 1] = o1;
            }
            if (sv.out) {
                sv.out[((size_t)s * CS + j) * 2] = o0;
                sv.out[((size_t)s * CS + j) * 2 + 1] = o1;
            }
        }
    }
    if (!dec) return;
    __syncthreads();
    // receiver mode: decisions, decision bytes and the window record (one warp)
    if (warp == 0) {
        const int NB = mq == 2 ? 1 : 2, BPS = 2 * NB;
        long long k0 = k_first + (long long)s * CS;
        int pwin = (int)(((long long)BPS * k0) % 32767);
        unsigned eA = 0, eB = 0, se = 0, nn = 0;
        for (int h = 0; h < 2; h++) {
            int q = lane + 32 * h;
            float vr = scale * os[2 * q], vi = scale * os[2 * q + 1];
            int LI = 0, LQ = 0;
            bool nr = false;
            for (int jj = 0; jj < mq - 1; jj++) {
                float th = (float)(2 * jj - (mq - 2));
                LI += vr >= th;
                LQ += vi >= th;
                nr |= fabsf(vr - th) < 1e-4f || fabsf(vi - th) < 1e-4f;
            }
            dec[(size_t)s * CS + q] = (uint8_t)(LI | (LQ << 3) | (nr ? 64 : 0));
            int pos = pwin + BPS * q;
            uint32_t w0 = prbs_bits[pos >> 5], w1 = prbs_bits[(pos >> 5) + 1];
            int ref = (int)(__funnelshift_l(w1, w0, pos & 31) >> (32 - BPS));
            for (int rq = 0; rq < 4; rq++) {
                int a = LI, bq = LQ;
                if (rq & 2) { a = mq - 1 - a; bq = mq - 1 - bq; }
                if (rq & 1) { int t = a; a = bq; bq = mq - 1 - t; }
                unsigned ne = __popc((((a ^ (a >> 1)) << NB) | (bq ^ (bq >> 1))) ^ ref);
                if (rq < 2) eA += ne << (16 * rq);
                else eB += ne << (16 * (rq - 2));
                se += (ne > 0) << (8 * rq);
            }
            nn += nr;
        }
        eA = warp_sum_i(eA);
        eB = warp_sum_i(eB);
        se = warp_sum_i(se);
        nn = warp_sum_i(nn);
        if (lane == 0) {
            winb[s] = 0;
            winrec[s] = make_uint4(eA, eB, se, nn << 8);
        }
    }
}

// shared-memory layout of the backward kernel (bytes)
struct BwdSmem {
    static constexpr int LDV = CH + 8;                           // padded rows of the MLP tiles (bf16)
    static constexpr int LDT = 152;                              // positions of duT (>= 144 + 8)
    static constexpr int LDH = 160;                              // positions of the transposed layer input
    static constexpr int NDU = 160;                              // rows of the padded du (8 zero rows first)
    static constexpr int X = 0;                                  // float [L0][2]
    static constexpr int DV = 1280;                              // float [S][64]
    static constexpr int DVB = DV + CS * CH * 4;                 // bf16 [S][LDV]   dv, rows j
    static constexpr int DVT = DVB + CS * LDV * 2;               // bf16 [64][LDV]  dv transposed, rows m
    static constexpr int H3T = DVT + CH * LDV * 2;               // bf16 [32][LDV]  h3 at the symbols, rows c
    static constexpr int M1T = H3T + CC * LDV * 2;               // bf16 [32][LDV]  M1 transposed, rows c
    static constexpr int DH = M1T + CC * LDV * 2;                // float [L1][32]  gradient of the layer output
    static constexpr int DUP = DH + L1 * CC * 4;                 // bf16 [NDU][32]  du from row 8 on
    static constexpr int DUT = DUP + NDU * CC * 2;               // bf16 [32][LDT]  du transposed
    static constexpr int HT0 = DUT + CC * LDT * 2;               // bf16 [32][LDH]  layer input transposed
    static constexpr int HT1 = HT0 + CC * LDH * 2;               // bf16 [32][LDH]  the same from position 1 on
    static constexpr int RED = HT1 + CC * LDH * 2;               // float [8][32]   bias partials
    static constexpr int TOTAL = RED + 8 * CC * 4;
};
static_assert(BwdSmem::TOTAL <= 113 * 1024, "two backward CTAs per SM");
static_assert(L1 + 8 <= BwdSmem::LDT && L1 + 16 <= BwdSmem::NDU && L0 <= BwdSmem::LDH,
              "padded tiles cover the largest layer");

// one m16n8k16 BF16 product: D += A * B with A row-major (row stride lda elements,
// even) and B given by its transpose Bt, row-major (row stride ldb, even)
__device__ __forceinline__ void mma_tile(float (&d)[4], const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *Bt,
                                         int ldb, int g, int tq)
{
    uint32_t a[4];
    a[0] = *reinterpret_cast<const uint32_t *>(A + lda * g + 2 * tq);
    a[1] = *reinterpret_cast<const uint32_t *>(A + lda * (g + 8) + 2 * tq);
    a[2] = *reinterpret_cast<const uint32_t *>(A + lda * g + 2 * tq + 8);
    a[3] = *reinterpret_cast<const uint32_t *>(A + lda * (g + 8) + 2 * tq + 8);
    mma_bf16(d, a, *reinterpret_cast<const uint32_t *>(Bt + ldb * g + 2 * tq),
             *reinterpret_cast<const uint32_t *>(Bt + ldb * g + 2 * tq + 8));
}

// Backward pass of one segment per CTA (256 threads): per-segment partial gradient
// gpart[s][NPRM].  The contractions run on the tensor cores with BF16 operands and
// FP32 accumulation (mma.sync m16n8k16): the MLP's dM1 and the gradient at the
// layer-3 output; per convolution layer 3 and 2 the weight gradient (K = the
// positions) and the input gradient (the forward's convolution over the zero-padded
// du with the tap-flipped, transposed weights wdT).  Elementwise steps (GELU
// derivatives, dM2, biases) and the 2-channel layer 1 stay in FP32.
__global__ void __launch_bounds__(256)
    k_cnn_bwd(const float *__restrict__ prm, const __nv_bfloat16 *__restrict__ wdT, const float2 *__restrict__ y,
              const long long *__restrict__ seg_start, const float *__restrict__ tgt, CnnSave sv, float norm,
              float *__restrict__ gpart)
{
    extern __shared__ __align__(16) unsigned char sm[];
    float *xs = reinterpret_cast<float *>(sm + BwdSmem::X);
    float *dv = reinterpret_cast<float *>(sm + BwdSmem::DV);
    __nv_bfloat16 *dvb = reinterpret_cast<__nv_bfloat16 *>(sm + BwdSmem::DVB);
    __nv_bfloat16 *dvt = reinterpret_cast<__nv_bfloat16 *>(sm + BwdSmem::DVT);
    __nv_bfloat16 *h3t = reinterpret_cast<__nv_bfloat16 *>(sm + BwdSmem::H3T);
    __nv_bfloat16 *m1t = reinterpret_cast<__nv_bfloat16 *>(sm + BwdSmem::M1T);
    float *dh = reinterpret_cast<float *>(sm + BwdSmem::DH);
    __nv_bfloat16 *dup = reinterpret_cast<__nv_bfloat16 *>(sm + BwdSmem::DUP);
    __nv_bfloat16 *dut = reinterpret_cast<__nv_bfloat16 *>(sm + BwdSmem::DUT);
    __nv_bfloat16 *ht0 = reinterpret_cast<__nv_bfloat16 *>(sm + BwdSmem::HT0);
    __nv_bfloat16 *ht1 = reinterpret_cast<__nv_bfloat16 *>(sm + BwdSmem::HT1);
    float *red = reinterpret_cast<float *>(sm + BwdSmem::RED);
    constexpr int LDV = BwdSmem::LDV, LDT = BwdSmem::LDT, LDH = BwdSmem::LDH, NDU = BwdSmem::NDU;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, tq = lane & 3;
    const int s = blockIdx.x;
    const __nv_bfloat16 bz = __float2bfloat16(0.f);
    float *G = gpart + (size_t)s * NPRM;
    const long long st = seg_start[s];
    for (int i = tid; i < L0; i += nth) {
        float2 v = y[st + i];
        xs[2 * i] = v.x;
        xs[2 * i + 1] = v.y;
    }
    const __nv_bfloat16 *h3 = sv.h3 + (size_t)s * L3 * CC;
    // ---- MLP head: dv = (dout . M2) gelu'(v) in FP32, bf16 copies for the products
    for (int i = tid; i < CS * CH; i += nth) {
        int j = i / CH, m = i - CH * j;
        float o0 = sv.out[((size_t)s * CS + j) * 2], o1 = sv.out[((size_t)s * CS + j) * 2 + 1];
        float d0 = 2.f * (o0 - tgt[((size_t)s * CS + j) * 2]) * norm;
        float d1 = 2.f * (o1 - tgt[((size_t)s * CS + j) * 2 + 1]) * norm;
        float vv = sv.v[((size_t)s * CS + j) * CH + m];
        float dz = d0 * prm[OM2 + m] + d1 * prm[OM2 + CH + m];
        float d = dz * gelu_df(vv);
        dv[i] = d;
        dvb[j * LDV + m] = __float2bfloat16(d);
        dvt[m * LDV + j] = __float2bfloat16(d);
    }
    for (int i = tid; i < CC * CS; i += nth) {   // h3 at the symbol positions, transposed
        int c = i / CS, j = i - CS * c;
        h3t[c * LDV + j] = h3[(2 * j) * CC + c];
    }
    for (int i = tid; i < CC * CH; i += nth) {   // M1 transposed, bf16
        int c = i / CH, m = i - CH * c;
        m1t[c * LDV + m] = __float2bfloat16(prm[OM1 + m * CC + c]);
    }
    for (int i = tid; i < L3 * CC; i += nth)     // odd positions of h3 feed nothing
        if ((i >> 5) & 1) dh[i] = 0.f;
    __syncthreads();
    // dM2, dc2 (z recomputed from v) and dc1 in FP32
    for (int i = tid; i < 2 * CH + 2 + CH; i += nth) {
        float a = 0.f;
        if (i < 2 * CH + 2) {
            const int oc = i < 2 * CH ? i / CH : i - 2 * CH;
            for (int j = 0; j < CS; j++) {
                float o = sv.out[((size_t)s * CS + j) * 2 + oc];
                float d = 2.f * (o - tgt[((size_t)s * CS + j) * 2 + oc]) * norm;
                a += (i < 2 * CH) ? d * gelu_f(sv.v[((size_t)s * CS + j) * CH + (i % CH)]) : d;
            }
            G[OM2 + i] = a;   // OC2 follows OM2 contiguously
        } else {
            const int m = i - (2 * CH + 2);
            for (int j = 0; j < CS; j++) a += dv[j * CH + m];
            G[OC1 + m] = a;
        }
    }
    // tiles 0..15: dM1[m][c] = sum_j dv[j][m] h3[2j][c]   (M = 64 m, N = 32 c, K = 64 j)
    // tiles 16..31: dh3[2j][c] = sum_m M1[m][c] dv[j][m]   (M = 64 j, N = 32 c, K = 64 m)
    for (int tile = warp; tile < 32; tile += 8) {
        const bool second = tile >= 16;
        const int mt = (tile & 15) >> 2, nt = tile & 3;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const __nv_bfloat16 *A = (second ? dvb : dvt) + LDV * 16 * mt;
        const __nv_bfloat16 *Bt = (second ? m1t : h3t) + LDV * 8 * nt;
#pragma unroll
        for (int k0 = 0; k0 < 64; k0 += 16) mma_tile(acc, A + k0, LDV, Bt + k0, LDV, g, tq);
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int r = 16 * mt + g + 8 * (i >> 1), c = 8 * nt + 2 * tq + (i & 1);
            if (second) dh[(2 * r) * CC + c] = acc[i];
            else G[OM1 + r * CC + c] = acc[i];
        }
    }
    __syncthreads();
    // ---- convolution layers 3 and 2 on the tensor cores, layer 1 in FP32
    for (int l = 3; l >= 1; l--) {
        const int Lout = (l == 3) ? L3 : (l == 2) ? L2 : L1;
        const int Lin = Lout + 8;
        const float *U = (l == 3) ? sv.u3 + (size_t)s * L3 * CC : (l == 2) ? sv.u2 + (size_t)s * L2 * CC
                                                                          : sv.u1 + (size_t)s * L1 * CC;
        const int OW = (l == 3) ? OW3 : (l == 2) ? OW2 : OW1, OB = (l == 3) ? OB3 : (l == 2) ? OB2 : OB1;
        // du = dh gelu'(u) for positions p < Lout (zero beyond): bias partials in FP32,
        // bf16 copies padded (dup: row p + 8) and transposed (dut); layer 1 in place
        float bsum = 0.f;
        for (int i = tid; i < LDT * CC; i += nth) {   // thread tid always holds channel tid & 31
            const int p = i >> 5, o = i & 31;
            const float d = p < Lout ? dh[p * CC + o] * gelu_df(U[p * CC + o]) : 0.f;
            bsum += d;
            if (l > 1) {
                dut[o * LDT + p] = __float2bfloat16(d);
                if (p + 8 < NDU) dup[(p + 8) * CC + o] = __float2bfloat16(d);
            } else if (p < Lout) {
                dh[p * CC + o] = d;
            }
        }
        red[warp * CC + lane] = bsum;
        if (l > 1) {
            for (int i = tid; i < 8 * CC; i += nth) dup[i] = bz;
            // layer input (h2 for layer 3, h1 for layer 2) transposed, zero beyond Lin
            const __nv_bfloat16 *src = (l == 3) ? sv.h2 + (size_t)s * L2 * CC : sv.h1 + (size_t)s * L1 * CC;
            for (int i = tid; i < CC * LDH; i += nth) {
                const int c = i / LDH, q = i - LDH * c;
                ht0[i] = q < Lin ? src[q * CC + c] : bz;
                ht1[i] = q + 1 < Lin ? src[(q + 1) * CC + c] : bz;
            }
        }
        __syncthreads();
        if (tid < CC) {
            float a = 0.f;
            for (int w = 0; w < 8; w++) a += red[w * CC + tid];
            G[OB + tid] = a;
        }
        if (l > 1) {
            // weight gradient dW[o][t][c] = sum_p du[p][o] h_in[p + t][c]: M = 32 (o),
            // N = 288 (t, c), K = 144 (p; du is zero from Lout on)
            for (int tile = warp; tile < 2 * 36; tile += 8) {
                const int mt = tile / 36, nt = tile - 36 * mt, t = nt >> 2, c0 = 8 * (nt & 3);
                // 32-bit loads need an even start: odd taps read the copy shifted by one
                const __nv_bfloat16 *Bt = ((t & 1) ? ht1 + (t - 1) : ht0 + t) + LDH * c0;
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 3
                for (int k0 = 0; k0 < 144; k0 += 16) mma_tile(acc, dut + LDT * 16 * mt + k0, LDT, Bt + k0, LDH, g, tq);
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int o = 16 * mt + g + 8 * (i >> 1), n = 8 * nt + 2 * tq + (i & 1);
                    G[OW + o * KW + n] = acc[i];
                }
            }
            // input gradient dh_in[q][c] = sum_t sum_o W[o][t][c] du[q - t][o]: row q of the
            // A operand is the padded du from row q on (tap t' = 8 - t at row q + t'); dh
            // (this layer's output gradient) was consumed above, so it takes dh_in
            const __nv_bfloat16 *Wt = wdT + (size_t)(l == 3 ? 1 : 0) * CC * KW;
            for (int tile = warp; tile < 9 * 4; tile += 8) {
                const int mt = tile >> 2, nt = tile & 3;
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
                for (int k0 = 0; k0 < KW; k0 += 16) {
                    uint32_t a[4];
                    const __nv_bfloat16 *ar = dup + CC * (16 * mt + g) + k0 + 2 * tq;
                    a[0] = *reinterpret_cast<const uint32_t *>(ar);
                    a[1] = *reinterpret_cast<const uint32_t *>(ar + CC * 8);
                    a[2] = *reinterpret_cast<const uint32_t *>(ar + 8);
                    a[3] = *reinterpret_cast<const uint32_t *>(ar + CC * 8 + 8);
                    const __nv_bfloat16 *br = Wt + KW * (8 * nt + g) + k0 + 2 * tq;
                    mma_bf16(acc, a, __ldg(reinterpret_cast<const unsigned int *>(br)),
                             __ldg(reinterpret_cast<const unsigned int *>(br + 8)));
                }
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int q = 16 * mt + g + 8 * (i >> 1), c = 8 * nt + 2 * tq + (i & 1);
                    if (q < Lin) dh[q * CC + c] = acc[i];
                }
            }
        } else {
            // layer 1 (2 input channels) in FP32: dW1[o][t][c] = sum_p du1[p][o] x[p + t][c]
            for (int i = tid; i < CC * CK * 2; i += nth) {
                int o = i / (CK * 2), r = i - o * CK * 2, t = r / 2, c = r - 2 * t;
                float a = 0.f;
                for (int p = 0; p < Lout; p++) a = fmaf(dh[p * CC + o], xs[(p + t) * 2 + c], a);
                G[OW + i] = a;
            }
        }
        __syncthreads();
    }
}

// grad[i] = sum_s gpart[s][i] (fixed order)
__global__ void k_cnn_reduce(const float *__restrict__ gpart, int nseg, float *__restrict__ grad)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPRM) return;
    float a = 0.f;
    for (int s = 0; s < nseg; s++) a += gpart[(size_t)s * NPRM + i];
    grad[i] = a;
}

// sum of the per-symbol squared errors (loss), fixed order within one CTA
__global__ void k_cnn_loss(const float *__restrict__ out, const float *__restrict__ tgt, long long n, float norm,
                           float *__restrict__ loss)
{
    __shared__ float red[256];
    float a = 0.f;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        float d = out[i] - tgt[i];
        a = fmaf(d, d, a);
    }
    red[threadIdx.x] = a;
    __syncthreads();
    for (int s2 = 128; s2 > 0; s2 >>= 1) {
        if ((int)threadIdx.x < s2) red[threadIdx.x] += red[threadIdx.x + s2];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] * norm;
}

// BF16 copy of a weight of layer 2 or 3 in the layout the backward input gradient
// reads: wdT[layer - 2][c][(8 - t) 32 + o] = W[o][t][c]
__device__ __forceinline__ void put_wdt(__nv_bfloat16 *wdT, int i, float w)
{
    const int lay = (i >= OW2 && i < OW2 + CC * KW) ? 0 : (i >= OW3 && i < OW3 + CC * KW) ? 1 : -1;
    if (lay < 0) return;
    const int rel = i - (lay ? OW3 : OW2), o = rel / KW, t = (rel % KW) / CC, c = rel % CC;
    wdT[(size_t)lay * CC * KW + c * KW + (CK - 1 - t) * CC + o] = __float2bfloat16(w);
}

// Adam on the FP32 master weights; refreshes the BF16 copies
__global__ void k_cnn_adam(float *__restrict__ prm, __nv_bfloat16 *__restrict__ prm_bf, __nv_bfloat16 *__restrict__ wdT,
                           float *__restrict__ m, float *__restrict__ v, const float *__restrict__ grad, float lr,
                           float b1t, float b2t)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPRM) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float g = grad[i];
    float mi = b1 * m[i] + (1.f - b1) * g, vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    float mh = mi / (1.f - b1t), vh = vi / (1.f - b2t);
    float w = prm[i] - lr * mh / (sqrtf(vh) + eps);
    prm[i] = w;
    prm_bf[i] = __float2bfloat16(w);
    put_wdt(wdT, i, w);
}

__global__ void k_cnn_tobf(const float *__restrict__ prm, __nv_bfloat16 *__restrict__ prm_bf,
                           __nv_bfloat16 *__restrict__ wdT)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NPRM) {
        prm_bf[i] = __float2bfloat16(prm[i]);
        put_wdt(wdT, i, prm[i]);
    }
}

// ====================================================================
// Receiver inference on the fifth-generation tensor cores (tcgen05).
//
// Tiles of kTS = 128 symbols (two 64-symbol windows).  One persistent CTA per SM
// runs kRxGroups independent groups of 8 warps, each with its own tile loop,
// activation planes, mbarrier, 128 tensor-memory columns and named barrier, and all
// reading the weights staged once per CTA: while one group waits on its MMAs or its
// tensor-memory loads, the others issue, so kRxGroups tiles are in flight per SM.  In
// a group two warps share each tensor-memory lane quarter, each taking half of the
// accumulator columns.  Activations live
// in shared memory as "planes" of 8 channels, each position one 16-byte row: with
// this layout the im2col operand of a 32-channel, 9-tap convolution at K-step ks
// (tap ks/2, channel groups 2 (ks % 2) and +1) is the plane pair read from
// position p + ks/2 onwards, i.e. a K-major no-swizzle matrix descriptor whose
// start address moves by whole 16-byte rows; no im2col copy is made.
//   layer 1 (2 -> 32, K = 18 padded to 32): one FP16 plane whose row p holds the
//      8 reals of positions p .. p+3; a descriptor whose two K core matrices sit
//      4 rows apart (leading offset 64 bytes) reads rows p, p+4 (K 0..15) and,
//      8 rows on, p+8, p+12 (K 16..31): the whole im2col row of position p;
//   layer 2 (32 -> 32): 18 tcgen05.mma (M = 128, N = 32, K = 16) per 128
//      positions; its epilogue stores the even and the odd positions in two
//      separate plane sets;
//   layer 3 (32 -> 32) only at the symbol (even) positions 2j: tap 2e reads the
//      even set from row j + e, tap 2e + 1 the odd set from row j + e, so one
//      M = 128 tile covers the tile's 128 symbols;
//   MLP 32 -> 64 (M = 128, N = 64) on the symbols, bias + GELU into FP16
//      planes, then 64 -> 2 as one more MMA (N = 16, two live columns);
//   decisions and window records as the FIR receiver.
// Inference precision: BF16 operands by default, FP16 as the alternative
// (activations and weights, converted from the FP32 master weights), FP32
// accumulation in tensor memory; bias and GELU in the same packed type, GELU by its
// tanh form 0.5 u (1 + tanh(sqrt(2/pi) (u + 0.044715 u^3))) with the hardware tanh
// (tanh.approx.bf16x2 / .f16x2): its distance to the erf form (< 2.2e-4 absolute)
// stays below the resolution the activations are stored with (2^-8 / 2^-11).
constexpr int kTS = 128;
constexpr int kP0 = 2 * kTS + 24, kP1 = kP0 - 8, kP2 = kP1 - 8;   // 280 272 264 input / layer-1 / layer-2 positions
constexpr int kMT1 = (kP1 + 127) / 128, kMT2 = (kP2 + 127) / 128;  // 3, 3 row tiles
constexpr int kRX = 128 * kMT1 + 12;         // rows of the layer-1 input plane (396)
constexpr int kR1 = 128 * kMT2 + 8;          // rows of the h1 planes (rows >= kP1 stay zero); h3 reuses rows < 128
constexpr int kRE = kP2 / 2 + 4;             // rows of each even / odd h2 plane (136; rows < 132 written)
constexpr int kWinT = kTS / 64;              // windows per tile
constexpr int kRxGroups = 4;                 // tile groups per CTA (tiles in flight per SM)
constexpr int kRxGroupThreads = 256;         // 8 warps: two per tensor-memory lane quarter
constexpr int kRxThreads = kRxGroups * kRxGroupThreads;
constexpr uint32_t kRxTmemGroup = 128;       // accumulator columns of one group
constexpr uint32_t kRxTmem = 512;            // the CTA's allocation (a power of two)
constexpr uint32_t kColOut = 96;             // accumulator columns of the 64 -> 2 projection
static_assert(kRxGroups * kRxTmemGroup <= kRxTmem && kRxTmem <= 512, "tensor memory of one SM");
// Shared memory: the weights (read by every group), then one block per group.
struct RxSmem {
    static constexpr int W2 = 0;                          // fp16 planes [36][32 rows][16 B]
    static constexpr int W3 = W2 + 36 * 512;
    static constexpr int M1 = W3 + 36 * 512;              // fp16 planes [4][64 rows][16 B]
    static constexpr int M2 = M1 + 4 * 1024;              // fp16 planes [8][16 rows][16 B] (rows 0, 1 live)
    static constexpr int B1 = M2 + 8 * 256;               // fp16 planes [4][32 rows][16 B]
    static constexpr int BH = B1 + 4 * 512;               // half2 biases: layers 1..3 [3][16], MLP [32]
    static constexpr int C2 = BH + 80 * 4;                // float [2]: output bias
    static constexpr int GRP = (C2 + 16 + 1023) & ~1023;  // first group block
    // one group's block, offsets from its start
    static constexpr int H1 = 0;                          // fp16 planes [4][kR1][16 B] (h1, then h3)
    static constexpr int HX = H1 + 4 * kR1 * 16;          // the layer-1 input plane [kRX][16 B], then the
                                                          // even/odd h2 planes [2][4][kRE][16 B], then the
                                                          // hidden planes [8][128][16 B], then the outputs
                                                          // float [kTS][2]
    static constexpr int HXB = 2 * 4 * kRE * 16;
    static constexpr int XS = HX + HXB;                   // float2 [kP0]: the next tile's input (async copy)
    static constexpr int BAR = XS + kP0 * 8;              // mbarrier
    static constexpr int GROUP = (BAR + 16 + 127) & ~127;
    static constexpr int SLOT = GRP + kRxGroups * GROUP;  // tensor-memory base address
    static constexpr int TOTAL = SLOT + 16;
};
static_assert(kRX * 16 <= RxSmem::HXB && 8 * 128 * 16 <= RxSmem::HXB, "aliases of the HX region fit");
static_assert(RxSmem::TOTAL <= 227 * 1024, "one receiver CNN CTA per SM");
static_assert(2 * (kRE - 4) == kP2, "even / odd h2 rows cover the layer-2 positions");

// barrier of one group's 256 threads (named barrier id, 1 + group); the second form
// also returns whether pred held in every thread of the group
__device__ __forceinline__ void group_sync(int id)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(kRxGroupThreads) : "memory");
}
__device__ __forceinline__ bool group_and(int id, bool pred)
{
    uint32_t r;
    asm volatile("{\n .reg .pred q, o;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred o, %2, %3, q;\n"
                 " selp.u32 %0, 1, 0, o;\n}"
                 : "=r"(r)
                 : "r"((uint32_t)pred), "r"(id), "n"(kRxGroupThreads)
                 : "memory");
    return r != 0;
}

__device__ __forceinline__ uint32_t h2_bits(__half2 h) { return *reinterpret_cast<uint32_t *>(&h); }
__device__ __forceinline__ __half2 bits_h2(uint32_t u) { return *reinterpret_cast<__half2 *>(&u); }

__device__ __forceinline__ uint32_t b2_bits(__nv_bfloat162 h) { return *reinterpret_cast<uint32_t *>(&h); }
__device__ __forceinline__ __nv_bfloat162 bits_b2(uint32_t u) { return *reinterpret_cast<__nv_bfloat162 *>(&u); }

// two FP32 values as one packed 16-bit pair (round to nearest even): FP16 or BF16
template <bool BF>
__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    if constexpr (BF) return b2_bits(__floats2bfloat162_rn(a, b));
    else return h2_bits(__floats2half2_rn(a, b));
}

// bias + GELU of two FP32 accumulators in packed FP16 (tanh form, hardware tanh),
// returned doubled: u = acc + b; t = tanh(u (c0 + c1 u^2)); 2 GELU(u) = u (1 + t) =
// u + u t.  The layers that read these activations take their weights halved, so the
// products they accumulate are those of GELU(u) and the true weights: a factor of two
// commutes with rounding, so the result is that of the undoubled form (BF16; FP16
// where no value is subnormal) at one operation less per pair.
__device__ __forceinline__ uint32_t gelu_h2(uint32_t a, uint32_t b, uint32_t bias)
{
    const __half2 c0 = __float2half2_rn(0.7978845608028654f), c1 = __float2half2_rn(0.7978845608028654f * 0.044715f);
    const __half2 u = __hadd2(__floats2half2_rn(__uint_as_float(a), __uint_as_float(b)), bits_h2(bias));
    const __half2 arg = __hmul2(u, __hfma2(__hmul2(u, u), c1, c0));
    uint32_t th;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(th) : "r"(h2_bits(arg)));
    return h2_bits(__hfma2(u, bits_h2(th), u));
}
// the same in packed BF16
__device__ __forceinline__ uint32_t gelu_b2(uint32_t a, uint32_t b, uint32_t bias)
{
    const __nv_bfloat162 c0 = __float2bfloat162_rn(0.7978845608028654f),
                         c1 = __float2bfloat162_rn(0.7978845608028654f * 0.044715f);
    const __nv_bfloat162 u = __hadd2(__floats2bfloat162_rn(__uint_as_float(a), __uint_as_float(b)), bits_b2(bias));
    const __nv_bfloat162 arg = __hmul2(u, __hfma2(__hmul2(u, u), c1, c0));
    uint32_t th;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(th) : "r"(b2_bits(arg)));
    return b2_bits(__hfma2(u, bits_b2(th), u));
}
template <bool BF>
__device__ __forceinline__ uint32_t gelu2(uint32_t a, uint32_t b, uint32_t bias)
{
    if constexpr (BF) return gelu_b2(a, b, bias);
    else return gelu_h2(a, b, bias);
}

template <bool BF>
__global__ void __launch_bounds__(kRxThreads, 1)
    k_cnn_rx_tc(const float *__restrict__ prm, const float2 *__restrict__ y,
                long long seg_base, long long y_end, int nwin, uint8_t *__restrict__ dec, uint8_t *__restrict__ winb,
                uint4 *__restrict__ winrec, const uint32_t *__restrict__ prbs_bits, long long k_first, float scale,
                int mq, float2 *__restrict__ soft, int *err)
{
    extern __shared__ __align__(16) unsigned char sm[];   // no-swizzle operands: 16-byte rows
    unsigned char *sW2 = sm + RxSmem::W2, *sW3 = sm + RxSmem::W3, *sM1 = sm + RxSmem::M1, *sM2 = sm + RxSmem::M2;
    unsigned char *sB1 = sm + RxSmem::B1;
    uint32_t *bh = reinterpret_cast<uint32_t *>(sm + RxSmem::BH);   // half2 bias pairs
    float *c2 = reinterpret_cast<float *>(sm + RxSmem::C2);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + RxSmem::SLOT);
    const int tid = threadIdx.x, grp = tid / kRxGroupThreads, gtid = tid % kRxGroupThreads;
    const int lane = tid & 31, warp = tid >> 5, gwarp = gtid >> 5, quarter = gwarp & 3, ch = gwarp >> 2;
    const int gbar = 1 + grp;   // the group's named barrier
    unsigned char *gb = sm + RxSmem::GRP + grp * RxSmem::GROUP;
    unsigned char *sH1 = gb + RxSmem::H1, *sHX = gb + RxSmem::HX;
    float *os = reinterpret_cast<float *>(sHX);   // the outputs, after the hidden planes are consumed
    float2 *xs = reinterpret_cast<float2 *>(gb + RxSmem::XS);
    uint64_t *bar = reinterpret_cast<uint64_t *>(gb + RxSmem::BAR);
    constexpr int PL1 = kR1 * 16, PLE = kRE * 16, EO = 4 * PLE;

    if (gtid == 0) mbar_init(bar, 1);
    __syncwarp();
    if (warp == 0) tmem_alloc(tslot, kRxTmem);
    // weights: B operands as K-major planes (chunk (row n, K column kk) at kk * rows * 16 + n * 16)
    // 8 FP32 weights of a layer that reads GELU outputs -> 16 bytes of FP16 / BF16,
    // halved (the epilogues store 2 GELU(u))
    auto h8 = [&](const float *src) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; i++) w[i] = pack2<BF>(0.5f * src[2 * i], 0.5f * src[2 * i + 1]);
        return make_uint4(w[0], w[1], w[2], w[3]);
    };
    for (int u = tid; u < 36 * 32; u += kRxThreads) {
        int n = u & 31, kk = u >> 5;
        *reinterpret_cast<uint4 *>(sW2 + kk * 512 + n * 16) = h8(prm + OW2 + n * KW + 8 * kk);
        *reinterpret_cast<uint4 *>(sW3 + kk * 512 + n * 16) = h8(prm + OW3 + n * KW + 8 * kk);
    }
    for (int u = tid; u < 4 * CH; u += kRxThreads) {
        int n = u & 63, kk = u >> 6;
        *reinterpret_cast<uint4 *>(sM1 + kk * 1024 + n * 16) = h8(prm + OM1 + n * CC + 8 * kk);
    }
    for (int u = tid; u < 8 * 16; u += kRxThreads) {   // output projection: rows 0, 1 = the two outputs
        int n = u & 15, kk = u >> 4;
        *reinterpret_cast<uint4 *>(sM2 + kk * 256 + n * 16) =
            n < 2 ? h8(prm + OM2 + n * CH + 8 * kk) : make_uint4(0, 0, 0, 0);
    }
    for (int u = tid; u < 4 * 32; u += kRxThreads) {   // layer-1 weights, FP16, K padded to 32
        int n = u & 31, kk = u >> 5;
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            int k0 = 8 * kk + 2 * i;
            float a = k0 < 18 ? prm[OW1 + n * 18 + k0] : 0.f, b = k0 + 1 < 18 ? prm[OW1 + n * 18 + k0 + 1] : 0.f;
            w[i] = pack2<BF>(a, b);
        }
        *reinterpret_cast<uint4 *>(sB1 + kk * 512 + n * 16) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    for (int i = tid; i < 3 * 16; i += kRxThreads) {
        const int off = (i < 16 ? OB1 : i < 32 ? OB2 : OB3) + 2 * (i & 15);
        bh[i] = pack2<BF>(prm[off], prm[off + 1]);
    }
    for (int i = tid; i < 32; i += kRxThreads) bh[48 + i] = pack2<BF>(prm[OC1 + 2 * i], prm[OC1 + 2 * i + 1]);
    if (tid < 2) c2[tid] = prm[OC2 + tid];
    const int ntiles = (nwin + kWinT - 1) / kWinT;
    const int t0 = (int)blockIdx.x * kRxGroups + grp, tstep = (int)gridDim.x * kRxGroups;
    // a tile's input, copied asynchronously into the group's buffer (zero past the stream end)
    auto prefetch = [&](int t) {
        for (int i = gtid; i < kP0; i += kRxGroupThreads) {
            const long long g = seg_base + 2LL * kTS * t + i;
            cp_async8(xs + i, g < y_end ? y + g : y, g < y_end);
        }
        cp_async_commit();
    };
    if (t0 < ntiles) prefetch(t0);
    // rows past the computed positions are read by the last row tiles: zero once
    for (int i = gtid; i < 4 * kR1; i += kRxGroupThreads)
        *reinterpret_cast<uint4 *>(sH1 + (i / kR1) * PL1 + (i % kR1) * 16) = make_uint4(0, 0, 0, 0);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot + (uint32_t)grp * kRxTmemGroup;   // the group's columns
    constexpr uint32_t kFmt = BF ? 1u : 0u;   // kind::f16 operand format: F16 or BF16
    const uint32_t id16 = umma_idesc(kFmt, 128, 16), id32 = umma_idesc(kFmt, 128, 32), id64 = umma_idesc(kFmt, 128, 64);
    const uint32_t aB1 = smem_u32(sB1), aH1 = smem_u32(sH1), aHX = smem_u32(sHX), aW2 = smem_u32(sW2),
                   aW3 = smem_u32(sW3), aM1 = smem_u32(sM1), aM2 = smem_u32(sM2);
    const uint32_t tq = tmem + ((uint32_t)(32 * quarter) << 16);   // this warp's lane quarter
    // matrix descriptors at the operand bases; an operand offset of o bytes adds o >> 4
    // to the start-address field, so the issue loops add compile-time constants
    const uint64_t dX = umma_sdesc(aHX, 64, 128), dB1 = umma_sdesc(aB1, 512, 128);
    const uint64_t dH1 = umma_sdesc(aH1, PL1, 128), dW2 = umma_sdesc(aW2, 512, 128), dW3 = umma_sdesc(aW3, 512, 128);
    const uint64_t dEO = umma_sdesc(aHX, PLE, 128), dM1 = umma_sdesc(aM1, 1024, 128);
    const uint64_t dHid = umma_sdesc(aHX, 2048, 128), dM2 = umma_sdesc(aM2, 256, 128);
    unsigned phase = 0;
    bool ok = true;

    auto wait_mma = [&]() -> bool {
        bool done = mbar_wait(bar, phase);
        if (!done) {
            atomicExch(err, (int)RX_ETIMEOUT);
            mbar_wait(bar, phase);
        }
        phase ^= 1u;
        return group_and(gbar, done);
    };
    // conv epilogue of MT row tiles: rows of this warp's lane quarter, channel groups
    // 2 ch and 2 ch + 1 (8 channels each) one after the other, each with every row
    // tile's accumulator load in flight before one wait; row -> address of its
    // 16-byte FP16 row of channel group cq in the destination
    auto conv_epi = [&](auto mt, int valid, const uint32_t *bias, auto dst_row) {
        constexpr int MT = decltype(mt)::value;
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const int cq = 2 * ch + c;
            uint32_t r[8 * MT];
#pragma unroll
            for (int m = 0; m < MT; m++)
                tmem_ld8_nw(tq + 32 * m + 8 * cq, *reinterpret_cast<uint32_t(*)[8]>(r + 8 * m));
            tmem_wait_ld(r);
            const uint4 b = *reinterpret_cast<const uint4 *>(bias + 4 * cq);
#pragma unroll
            for (int m = 0; m < MT; m++) {
                const int row = 128 * m + 32 * quarter + lane;
                const uint32_t *q = r + 8 * m;
                if (row < valid)
                    *reinterpret_cast<uint4 *>(dst_row(row, cq)) =
                        make_uint4(gelu2<BF>(q[0], q[1], b.x), gelu2<BF>(q[2], q[3], b.y),
                                   gelu2<BF>(q[4], q[5], b.z), gelu2<BF>(q[6], q[7], b.w));
            }
        }
    };

    for (int t = t0; t < ntiles && ok; t += tstep) {
        // layer-1 input plane: row p = positions p .. p+3 (8 reals) in FP16, zero past kP0
        cp_async_wait_all();
        group_sync(gbar);   // the tile's input is in xs
        for (int p = gtid; p < kRX; p += kRxGroupThreads) {
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const float2 v = p + i < kP0 ? xs[p + i] : make_float2(0.f, 0.f);
                w[i] = pack2<BF>(v.x, v.y);
            }
            *reinterpret_cast<uint4 *>(sHX + p * 16) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        fence_async_smem();
        group_sync(gbar);
        if (t + tstep < ntiles) prefetch(t + tstep);   // lands while this tile computes
        if (gtid == 0) {
            tc_fence_after();
#pragma unroll
            for (int m = 0; m < kMT1; m++)
#pragma unroll
                for (int ks = 0; ks < 2; ks++)
                    umma_f16(tmem + 32 * m, dX + (((128 * m + 8 * ks) * 16) >> 4), dB1 + ((2 * ks * 512) >> 4), id32,
                             ks > 0);
            umma_commit(bar);
        }
        if (!(ok = wait_mma())) break;
        tc_fence_after();
        conv_epi(std::integral_constant<int, kMT1>(), kP1, bh,
                 [&](int row, int cq) { return sH1 + cq * PL1 + row * 16; });
        fence_async_smem();
        tc_fence_before();
        group_sync(gbar);
        // layer 2 (reads h1; the input plane is free)
        if (gtid == 0) {
            tc_fence_after();
#pragma unroll
            for (int m = 0; m < kMT2; m++)
#pragma unroll
                for (int ks = 0; ks < 18; ks++)
                    umma_f16(tmem + 32 * m, dH1 + (((128 * m + ks / 2) * 16 + 2 * (ks & 1) * PL1) >> 4),
                             dW2 + ((2 * ks * 512) >> 4), id32, ks > 0);
            umma_commit(bar);
        }
        if (!(ok = wait_mma())) break;
        tc_fence_after();
        conv_epi(std::integral_constant<int, kMT2>(), kP2, bh + 16,
                 [&](int row, int cq) { return sHX + (row & 1) * EO + cq * PLE + (row >> 1) * 16; });
        fence_async_smem();
        tc_fence_before();
        group_sync(gbar);
        // layer 3 at the symbol positions: tap d reads set d & 1 from row j + d / 2
        if (gtid == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < 18; ks++) {
                const int d = ks >> 1;
                umma_f16(tmem, dEO + (((d & 1) * EO + (d >> 1) * 16 + 2 * (ks & 1) * PLE) >> 4),
                         dW3 + ((2 * ks * 512) >> 4), id32, ks > 0);
            }
            umma_commit(bar);
        }
        if (!(ok = wait_mma())) break;
        tc_fence_after();
        conv_epi(std::integral_constant<int, 1>(), kTS, bh + 32,
                 [&](int row, int cq) { return sH1 + cq * PL1 + row * 16; });   // h3, row = symbol
        fence_async_smem();
        tc_fence_before();
        group_sync(gbar);
        // MLP 32 -> 64 on the symbols (M = 128, N = 64, K = 32)
        if (gtid == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < 2; ks++)
                umma_f16(tmem, dH1 + ((2 * ks * PL1) >> 4), dM1 + ((2 * ks * 1024) >> 4), id64, ks > 0);
            umma_commit(bar);
        }
        if (!(ok = wait_mma())) break;
        tc_fence_after();
#pragma unroll
        for (int c = 0; c < 2; c++) {
            // hidden units 16 hq .. + 15 of symbol row -> planes 2 hq, 2 hq + 1 (the h2 planes are free)
            const int hq = 2 * ch + c;
            uint32_t r[16];
            tmem_ld16(tq + 16 * hq, r);
            const int row = 32 * quarter + lane;
            const uint4 b0 = *reinterpret_cast<const uint4 *>(bh + 48 + 8 * hq);
            const uint4 b1 = *reinterpret_cast<const uint4 *>(bh + 48 + 8 * hq + 4);
            *reinterpret_cast<uint4 *>(sHX + (2 * hq) * 2048 + row * 16) =
                make_uint4(gelu2<BF>(r[0], r[1], b0.x), gelu2<BF>(r[2], r[3], b0.y), gelu2<BF>(r[4], r[5], b0.z),
                           gelu2<BF>(r[6], r[7], b0.w));
            *reinterpret_cast<uint4 *>(sHX + (2 * hq + 1) * 2048 + row * 16) =
                make_uint4(gelu2<BF>(r[8], r[9], b1.x), gelu2<BF>(r[10], r[11], b1.y), gelu2<BF>(r[12], r[13], b1.z),
                           gelu2<BF>(r[14], r[15], b1.w));
        }
        fence_async_smem();
        tc_fence_before();
        group_sync(gbar);
        // 64 -> 2 (M = 128, N = 16 with rows 2..15 of B zero, K = 64)
        if (gtid == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < 4; ks++)
                umma_f16(tmem + kColOut, dHid + ((2 * ks * 2048) >> 4), dM2 + ((2 * ks * 256) >> 4), id16, ks > 0);
            umma_commit(bar);
        }
        if (!(ok = wait_mma())) break;
        tc_fence_after();
        // the projection has read the hidden planes: the outputs take their place
        if (ch == 0) {
            uint32_t r[8];
            tmem_ld8(tq + kColOut, r);
            const int j = 32 * quarter + lane;
            const float o0 = __uint_as_float(r[0]) + c2[0], o1 = __uint_as_float(r[1]) + c2[1];
            os[2 * j] = o0;
            os[2 * j + 1] = o1;
            const long long ks = (long long)kTS * t + j;
            if (soft && ks < 64LL * nwin) soft[ks] = make_float2(o0, o1);
        }
        tc_fence_before();
        group_sync(gbar);
        // decisions and window records: warp w < kWinT of the group takes window kWinT t + w
        if (gwarp < kWinT && kWinT * t + gwarp < nwin) {
            const int s = kWinT * t + gwarp;
            const float *osw = os + 2 * 64 * gwarp;
            const int NB = mq == 2 ? 1 : 2, BPS = 2 * NB;
            long long k0 = k_first + (long long)s * CS;
            int pwin = (int)(((long long)BPS * k0) % 32767);
            unsigned eA = 0, eB = 0, se = 0, nn = 0;
            for (int h = 0; h < 2; h++) {
                int q = lane + 32 * h;
                float vr = scale * osw[2 * q], vi = scale * osw[2 * q + 1];
                int LI = 0, LQ = 0;
                bool nr = false;
                for (int jj = 0; jj < mq - 1; jj++) {
                    float th = (float)(2 * jj - (mq - 2));
                    LI += vr >= th;
                    LQ += vi >= th;
                    nr |= fabsf(vr - th) < 1e-4f || fabsf(vi - th) < 1e-4f;
                }
                dec[(size_t)s * CS + q] = (uint8_t)(LI | (LQ << 3) | (nr ? 64 : 0));
                int pos = pwin + BPS * q;
                uint32_t w0 = __ldg(prbs_bits + (pos >> 5)), w1w = __ldg(prbs_bits + (pos >> 5) + 1);
                int ref = (int)(__funnelshift_l(w1w, w0, pos & 31) >> (32 - BPS));
                for (int rq = 0; rq < 4; rq++) {
                    int a = LI, bq = LQ;
                    if (rq & 2) { a = mq - 1 - a; bq = mq - 1 - bq; }
                    if (rq & 1) { int tt = a; a = bq; bq = mq - 1 - tt; }
                    unsigned ne = __popc((((a ^ (a >> 1)) << NB) | (bq ^ (bq >> 1))) ^ ref);
                    if (rq < 2) eA += ne << (16 * rq);
                    else eB += ne << (16 * (rq - 2));
                    se += (ne > 0) << (8 * rq);
                }
                nn += nr;
            }
            eA = warp_sum_i(eA);
            eB = warp_sum_i(eB);
            se = warp_sum_i(se);
            nn = warp_sum_i(nn);
            if (lane == 0) {
                winb[s] = 0;
                winrec[s] = make_uint4(eA, eB, se, nn << 8);
            }
        }
        group_sync(gbar);   // the outputs are read before the next tile's input plane
    }
    cp_async_wait_all();   // a prefetch may still be in flight after an early exit
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(*tslot, kRxTmem);
}

cudaError_t prepare_cnn_rx()
{
    cudaError_t e = cudaFuncSetAttribute(k_cnn_rx_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, RxSmem::TOTAL);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cnn_rx_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, RxSmem::TOTAL);
    return e;
}

cudaError_t launch_cnn_decide(const float *prm, const float2 *y, long long seg_base, long long y_end,
                              int nwin, uint8_t *dec, uint8_t *winb, uint4 *winrec, const uint32_t *prbs_bits,
                              long long k_first, float scale, int mq, float2 *soft, int *err, int nsm, cudaStream_t st,
                              int bf16)
{
    if (nwin <= 0) return cudaSuccess;
    int ntiles = (nwin + kWinT - 1) / kWinT, nctas = (ntiles + kRxGroups - 1) / kRxGroups;
    unsigned grid = (unsigned)(nctas < nsm ? nctas : nsm);   // one persistent CTA per SM
    if (bf16)
        k_cnn_rx_tc<true><<<grid, kRxThreads, RxSmem::TOTAL, st>>>(prm, y, seg_base, y_end, nwin, dec, winb, winrec,
                                                                  prbs_bits, k_first, scale, mq, soft, err);
    else
        k_cnn_rx_tc<false><<<grid, kRxThreads, RxSmem::TOTAL, st>>>(prm, y, seg_base, y_end, nwin, dec, winb, winrec,
                                                                   prbs_bits, k_first, scale, mq, soft, err);
    return cudaGetLastError();
}

}  // namespace rxk

using namespace rxk;

struct rx_cnn {
    int max_seg;
    float *prm, *grad, *m, *v, *gpart, *loss;
    __nv_bfloat16 *prm_bf;
    __nv_bfloat16 *wdT;   // layer 2 and 3 weights for the backward input gradient
    CnnSave sv;
    long long step;
};

extern "C" {

int rx_cnn_nparams(void) { return NPRM; }

void rx_cnn_destroy(rx_cnn *c)
{
    if (!c) return;
    void *p[] = {c->prm, c->grad, c->m, c->v, c->gpart, c->loss, c->prm_bf, c->wdT, c->sv.u1, c->sv.u2, c->sv.u3,
                 c->sv.h1, c->sv.h2, c->sv.h3, c->sv.v, c->sv.out};
    for (void *q : p)
        if (q) cudaFree(q);
    free(c);
}

rx_status rx_cnn_create(int max_seg, rx_cnn **out)
{
    if (!out || max_seg <= 0) return RX_EINVAL;
    *out = nullptr;
    rx_cnn *c = (rx_cnn *)calloc(1, sizeof(rx_cnn));
    if (!c) return RX_ENOMEM;
    c->max_seg = max_seg;
    size_t S = (size_t)max_seg;
    struct {
        void **p;
        size_t b;
    } al[] = {{(void **)&c->prm, NPRM * 4},
              {(void **)&c->grad, NPRM * 4},
              {(void **)&c->m, NPRM * 4},
              {(void **)&c->v, NPRM * 4},
              {(void **)&c->gpart, S * NPRM * 4},
              {(void **)&c->loss, 16},
              {(void **)&c->prm_bf, NPRM * 2 + 64},
              {(void **)&c->wdT, 2 * CC * KW * 2},
              {(void **)&c->sv.u1, S * L1 * CC * 4},
              {(void **)&c->sv.u2, S * L2 * CC * 4},
              {(void **)&c->sv.u3, S * L3 * CC * 4},
              {(void **)&c->sv.h1, S * L1 * CC * 2},
              {(void **)&c->sv.h2, S * L2 * CC * 2},
              {(void **)&c->sv.h3, S * L3 * CC * 2},
              {(void **)&c->sv.v, S * CS * CH * 4},
              {(void **)&c->sv.out, S * CS * 2 * 4}};
    for (auto &a : al) {
        if (cudaMalloc(a.p, a.b) != cudaSuccess || cudaMemset(*a.p, 0, a.b) != cudaSuccess) {
            cudaGetLastError();
            rx_cnn_destroy(c);
            return RX_ENOMEM;
        }
    }
    cudaFuncSetAttribute(k_cnn_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, FwdSmem::TOTAL);
    cudaFuncSetAttribute(k_cnn_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, BwdSmem::TOTAL);
    *out = c;
    return RX_OK;
}

rx_status rx_cnn_set_params(rx_cnn *c, const float *host, int n)
{
    if (!c || !host || n != NPRM) return RX_EINVAL;
    if (cudaMemcpy(c->prm, host, NPRM * 4, cudaMemcpyHostToDevice) != cudaSuccess) return RX_ECUDA;
    cudaMemset(c->m, 0, NPRM * 4);
    cudaMemset(c->v, 0, NPRM * 4);
    c->step = 0;
    k_cnn_tobf<<<(NPRM + 255) / 256, 256>>>(c->prm, c->prm_bf, c->wdT);
    if (cudaDeviceSynchronize() != cudaSuccess) return RX_ECUDA;
    return RX_OK;
}

rx_status rx_cnn_get_params(rx_cnn *c, float *host, int n)
{
    if (!c || !host || n != NPRM) return RX_EINVAL;
    if (cudaMemcpy(host, c->prm, NPRM * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return RX_ECUDA;
    return RX_OK;
}

rx_status rx_cnn_forward(rx_cnn *c, const float *y, const int64_t *seg_start, int nseg, float *out, void *stream)
{
    if (!c || !y || !seg_start || !out || nseg <= 0) return RX_EINVAL;
    CnnSave sv;
    memset(&sv, 0, sizeof sv);
    k_cnn_fwd<<<nseg, kCnnThreads, FwdSmem::TOTAL, (cudaStream_t)stream>>>(
        c->prm, c->prm_bf, (const float2 *)y, (const long long *)seg_start, 0, 0, out, sv, nullptr, nullptr, nullptr,
        nullptr, 0, 1.f, 4);
    return cudaGetLastError() == cudaSuccess ? RX_OK : RX_ECUDA;
}

rx_status rx_cnn_grad(rx_cnn *c, const float *y, const int64_t *seg_start, const float *tgt, int nseg, float *grad_out,
                      float *loss_out, void *stream)
{
    if (!c || !y || !seg_start || !tgt || nseg <= 0 || nseg > c->max_seg) return RX_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    float norm = 1.f / ((float)nseg * CS);
    k_cnn_fwd<<<nseg, kCnnThreads, FwdSmem::TOTAL, st>>>(c->prm, c->prm_bf, (const float2 *)y,
                                                         (const long long *)seg_start, 0, 0, nullptr, c->sv, nullptr,
                                                         nullptr, nullptr, nullptr, 0, 1.f, 4);
    k_cnn_bwd<<<nseg, 256, BwdSmem::TOTAL, st>>>(c->prm, c->wdT, (const float2 *)y, (const long long *)seg_start,
                                                 tgt, c->sv, norm, c->gpart);
    k_cnn_reduce<<<(NPRM + 255) / 256, 256, 0, st>>>(c->gpart, nseg, c->grad);
    k_cnn_loss<<<1, 256, 0, st>>>(c->sv.out, tgt, (long long)nseg * CS * 2, norm, c->loss);
    if (grad_out) cudaMemcpyAsync(grad_out, c->grad, NPRM * 4, cudaMemcpyDeviceToDevice, st);
    if (loss_out) cudaMemcpyAsync(loss_out, c->loss, 4, cudaMemcpyDeviceToDevice, st);
    return cudaGetLastError() == cudaSuccess ? RX_OK : RX_ECUDA;
}

rx_status rx_cnn_adam_step(rx_cnn *c, float lr, void *stream)
{
    if (!c || !(lr > 0)) return RX_EINVAL;
    c->step++;
    float b1t = powf(0.9f, (float)c->step), b2t = powf(0.999f, (float)c->step);
    k_cnn_adam<<<(NPRM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(c->prm, c->prm_bf, c->wdT, c->m, c->v, c->grad,
                                                                     lr, b1t, b2t);
    return cudaGetLastError() == cudaSuccess ? RX_OK : RX_ECUDA;
}

// device pointers of the parameters (for the receiver's CNN path)
const float *rx_cnn_dev_params(const rx_cnn *c) { return c ? c->prm : nullptr; }

}  // extern "C"
