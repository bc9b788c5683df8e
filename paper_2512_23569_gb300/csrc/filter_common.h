// Pieces of the collaborative filter shared by its SIMT kernels (filter.cu)
// and its tensor-core kernel (filter_tc.cu): the Haar transform along the
// group axis (Eq. 8) and the exact fixed-point aggregation.
#pragma once

namespace hts {
namespace fc {

constexpr float R2F = 0.70710678118654752f;  // 1/sqrt(2)
constexpr float K3F = 0.57735026918962576f;  // 1/sqrt(3)
constexpr float S3H = 0.86602540378443865f;  // sqrt(3)/2
constexpr float K23F = 0.81649658092772604f;  // sqrt(2/3)

// --------------------------------------------------------- Haar (Eq. 8)

// Forward: output row order of Eq. 8 (row 0 = sum / sqrt K, then the
// coarse-to-fine difference rows, the finest K/2 differences last).
template <int K>
__device__ __forceinline__ void haar_fwd(float (&x)[K]) {
#pragma unroll
    for (int n = K; n >= 2; n >>= 1) {
        float t[K];
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            t[i] = (x[2 * i] + x[2 * i + 1]) * R2F;
            t[n / 2 + i] = (x[2 * i] - x[2 * i + 1]) * R2F;
        }
#pragma unroll
        for (int i = 0; i < n; ++i) x[i] = t[i];
    }
}

template <int K>
__device__ __forceinline__ void haar_inv(float (&x)[K]) {
#pragma unroll
    for (int n = 2; n <= K; n <<= 1) {
        float t[K];
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            t[2 * i] = (x[i] + x[n / 2 + i]) * R2F;
            t[2 * i + 1] = (x[i] - x[n / 2 + i]) * R2F;
        }
#pragma unroll
        for (int i = 0; i < n; ++i) x[i] = t[i];
    }
}

// Fixed-point aggregation: value * 2^16 rounded to int64 (|value| < 2^31).
__device__ __forceinline__ long long fix16(float v) { return __float2ll_rn(v * 65536.0f); }

// The same fixed-point value split as hi * 2^16 + lo, with |lo| <= 2^15 (fast
// path) or 0 <= lo < 2^16, for the tile's 32-bit shared sums.  For |v| < 2^22
// it needs no 64-bit conversion: adding 1.5 * 2^23 rounds to the nearest
// integer (ties to even) and leaves it in the low mantissa bits, for the
// integer part and again for the 16-bit fraction; both steps are exact, so
// hi * 2^16 + lo == fix16(v).
__device__ __forceinline__ void fix16_split(float v, int &hi, int &lo) {
    constexpr float MAGIC = 12582912.0f;  // 1.5 * 2^23
    constexpr int MAGIC_BITS = 0x4B400000;
    if (fabsf(v) < 4194304.0f) {
        const float t = v + MAGIC;
        hi = __float_as_int(t) - MAGIC_BITS;
        const float f = v - (t - MAGIC);  // v - round(v), exact
        lo = __float_as_int(fmaf(f, 65536.0f, MAGIC)) - MAGIC_BITS;
    } else {
        const long long q = fix16(v);
        hi = (int)(q >> 16);
        lo = (int)(q & 0xffff);
    }
}

}  // namespace fc
}  // namespace hts
