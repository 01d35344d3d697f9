// Self-check of the integer-pipe binary32 <-> binary64 conversions of common.cuh (widen_f32,
// narrow_f64, split_f64) against the hardware conversions, for msc_selftest_conversions.  A test
// helper: it allocates a 4-byte counter and synchronises the device.
#pragma once

#include "common.cuh"

namespace {
__device__ unsigned int conv_mix(unsigned long long& s) {  // splitmix64 step, high half
    s += 0x9e3779b97f4a7c15ull;
    unsigned long long z = s;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return (unsigned int)((z ^ (z >> 31)) >> 32);
}

// split_f64's reference: hi = RN(x), lo = RN(x - hi) with the difference formed exactly in binary64
// (hi has 24 significant bits inside x's binary64 grid), lo dropped where x's binary64 ulp lies
// below 2^-126 (|x| < 2^-74)
__device__ bool split_matches(double d) {
    float hi, lo;
    msc::split_f64(d, hi, lo);
    const float hr = __double2float_rn(d);
    if (__float_as_uint(hi) != __float_as_uint(hr)) return false;
    const unsigned int e = (unsigned int)(((unsigned long long)__double_as_longlong(d) >> 52) & 0x7ffu);
    if (isinf(hr)) return true;  // rounded up past the binary32 range: lo is not meaningful
    if (e - 897u > 253u || (int)e - 948 < 1) return lo == 0.0f;
    const float lr = __double2float_rn(d - (double)hr);
    return lo == lr && (lo != 0.0f || __float_as_uint(lo) == 0u);
}

__global__ void k_conversion_check(unsigned long long seed, int per_thread, unsigned int* bad) {
    unsigned long long s = seed ^ (0x5851f42d4c957f2dull * (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x));
    unsigned int nbad = 0;
    for (int i = 0; i < per_thread; ++i) {
        // random binary32 patterns (every exponent) and random binary64 patterns near the binary32 range
        const unsigned int fb = conv_mix(s);
        const float f = __uint_as_float(fb);
        const double w = msc::widen_f32(f), wr = (double)f;
        if (!(w == wr || (w != w && wr != wr)) || (w == wr && __double_as_longlong(w) != __double_as_longlong(wr))) ++nbad;
        const unsigned long long hi = conv_mix(s), lo = conv_mix(s);
        unsigned long long db = (hi << 32) | lo;
        const unsigned long long ex = 880ull + (hi % 290ull);  // exponents 880 .. 1169 around the range
        db = (db & 0x800fffffffffffffull) | (ex << 52);
        if ((i & 7) == 0) db = (db & ~0x1fffffffull) | ((i & 8) ? 0x10000000ull : 0x0fffffffull);  // ties, near ties
        if ((i & 15) == 4) db |= 0x000fffffe0000000ull;  // mantissa all ones above the cut: carries into the exponent
        const double d = __longlong_as_double((long long)db);
        const float n = msc::narrow_f64(d), nr = __double2float_rn(d);
        if (__float_as_uint(n) != __float_as_uint(nr)) ++nbad;
        if (!split_matches(d)) ++nbad;
    }
    if (nbad) atomicAdd(bad, nbad);
}
}  // namespace

extern "C" int msc_selftest_conversions(int blocks, int per_thread, unsigned long long seed, int* mismatches) {
    if (blocks < 1 || per_thread < 1 || !mismatches) return MSC_ERR_ARG;
    unsigned int* d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned int)) != cudaSuccess) return MSC_ERR_CUDA;
    unsigned int h = 0;
    if (cudaMemset(d, 0, sizeof(unsigned int)) != cudaSuccess) { cudaFree(d); return MSC_ERR_CUDA; }
    k_conversion_check<<<blocks, 256>>>(seed, per_thread, d);
    const bool ok = cudaGetLastError() == cudaSuccess &&
                    cudaMemcpy(&h, d, sizeof(unsigned int), cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(d);
    if (!ok) return MSC_ERR_CUDA;
    *mismatches = (int)h;
    return MSC_OK;
}
