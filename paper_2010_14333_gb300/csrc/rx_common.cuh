// Device helpers shared by the receiver kernels: complex arithmetic and the
// in-register 16-point DFT used by the radix-16 FFT passes.
#pragma once

#include <cuda_runtime.h>

namespace rxk {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// the hardware square-root approximation (positive normal x)
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// 4-point DFT in place; forward kernel e^{-2 pi i nk/4} (INV: e^{+...}, unscaled)
template <bool INV>
__device__ __forceinline__ void dft4(float2 &a, float2 &b, float2 &c, float2 &d)
{
    float2 s0 = cadd(a, c), s1 = csub(a, c), s2 = cadd(b, d), s3 = csub(b, d);
    a = cadd(s0, s2);
    c = csub(s0, s2);
    if (!INV) {   // X1 = s1 - j s3, X3 = s1 + j s3
        b = make_float2(s1.x + s3.y, s1.y - s3.x);
        d = make_float2(s1.x - s3.y, s1.y + s3.x);
    } else {      // X1 = s1 + j s3, X3 = s1 - j s3
        b = make_float2(s1.x - s3.y, s1.y + s3.x);
        d = make_float2(s1.x + s3.y, s1.y - s3.x);
    }
}

// W16^m = e^{-2 pi i m / 16} for m = 0..9 (the products q0*k1 of a 4x4 split)
__device__ __forceinline__ float2 w16(int m)
{
    const float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, r2 = 0.70710678118654752f;
    switch (m) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return make_float2(c1, -s1);
    case 2: return make_float2(r2, -r2);
    case 3: return make_float2(s1, -c1);
    case 4: return make_float2(0.f, -1.f);
    case 6: return make_float2(-r2, -r2);
    default: return make_float2(-c1, s1);   // m = 9
    }
}

// 16-point DFT of x[0..15] in registers, natural order in and out, unscaled.
// Split q = q0 + 4 q1, k = k1 + 4 k0: 4-point DFTs over q1, twiddle W16^(q0 k1),
// 4-point DFTs over q0.
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&x)[16])
{
#pragma unroll
    for (int q0 = 0; q0 < 4; q0++) dft4<INV>(x[q0], x[q0 + 4], x[q0 + 8], x[q0 + 12]);
#pragma unroll
    for (int q0 = 1; q0 < 4; q0++) {
#pragma unroll
        for (int k1 = 1; k1 < 4; k1++) {
            float2 w = w16(q0 * k1);
            if (INV) w.y = -w.y;
            x[q0 + 4 * k1] = cmul(x[q0 + 4 * k1], w);
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++) dft4<INV>(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
    // position 4 k1 + k0 now holds X[k1 + 4 k0]: transpose the 4x4 grid
    float2 t[16];
#pragma unroll
    for (int i = 0; i < 16; i++) t[i] = x[i];
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++)
#pragma unroll
        for (int k0 = 0; k0 < 4; k0++) x[k1 + 4 * k0] = t[4 * k1 + k0];
}

// ------------------------------------------------------------ packed FP32 pairs
// Two FP32 values in one 64-bit register, operated on by the sm_100-family paired
// FP32 instructions (fma.rn.f32x2 and friends): each half is an IEEE round-to-
// nearest operation, identical to the scalar one, at one instruction per pair.
typedef unsigned long long f2x;
__device__ __forceinline__ f2x f2_pack(float a, float b)
{
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(f2x v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ f2x f2_fma(f2x a, f2x b, f2x c)
{
    f2x d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2x f2_mul(f2x a, f2x b)
{
    f2x d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x f2_add(f2x a, f2x b)
{
    f2x d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// padded shared-memory index: one spare element per 16 avoids bank conflicts
// in the stride-16 radix-16 pass
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

__device__ __forceinline__ int warp_sum_i(int v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace rxk
