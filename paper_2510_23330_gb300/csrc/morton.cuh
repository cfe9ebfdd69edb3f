// morton.cuh -- root box and Morton keys (tree construction, Sec. 3.4 and
// 5.2.2 of Hirashima et al., SC'25), shared by the context path (sort.cu)
// and the allocation-free entry point (noalloc.cu) so that both compute the
// same keys from the same device code.
//
// Root box: lo_k = min x_k, ext = max_k(max x_k - lo_k), L = 2^ceil(log2 ext)
// (L = 1 when ext = 0), unit = L / 2^21.  Cell c_k = min(floor((x_k - lo_k) *
// 2^21 / L), 2^21 - 1) from exact FP64 operations; the key interleaves bit b
// of c_x, c_y, c_z at 3b+2, 3b+1, 3b.
#pragma once

#include <stdint.h>

#ifndef GNB_GRID_MAX
#define GNB_GRID_MAX 2097151
#endif

namespace gnb {

// Order-preserving map of a double to an unsigned integer (for atomic min/max).
__device__ __forceinline__ unsigned long long dbl_to_ord(double v)
{
    long long b = __double_as_longlong(v);
    return b >= 0 ? ((unsigned long long)b ^ 0x8000000000000000ull) : ~(unsigned long long)b;
}
__device__ __forceinline__ double ord_to_dbl(unsigned long long o)
{
    long long b = (o & 0x8000000000000000ull) ? (long long)(o ^ 0x8000000000000000ull) : (long long)~o;
    return __longlong_as_double(b);
}

// mm[0..2] = ordered minima, mm[3..5] = maxima, mm[6] = non-finite flag.
__device__ __forceinline__ void minmax_init(unsigned long long *mm, int t)
{
    if (t < 3) mm[t] = ~0ull;
    else if (t < 7) mm[t] = 0ull;
}

// Grid-stride min/max of the three coordinates; one atomic per warp and axis.
__device__ __forceinline__ void minmax_accumulate(const double *__restrict__ x, const double *__restrict__ y,
                                                  const double *__restrict__ z, int n, unsigned long long *mm)
{
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0, 0, 0};
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v[3] = {x[i], y[i], z[i]};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            bad |= !isfinite(v[a]);
            unsigned long long o = dbl_to_ord(v[a]);
            mn[a] = o < mn[a] ? o : mn[a];
            mx[a] = o > mx[a] ? o : mx[a];
        }
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long p = __shfl_xor_sync(0xffffffffu, mn[a], o);
            unsigned long long q = __shfl_xor_sync(0xffffffffu, mx[a], o);
            mn[a] = p < mn[a] ? p : mn[a];
            mx[a] = q > mx[a] ? q : mx[a];
        }
    }
    bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            atomicMin(&mm[a], mn[a]);
            atomicMax(&mm[3 + a], mx[a]);
        }
        if (bad) atomicExch(&mm[6], 1ull);
    }
}

// box = {lo_x, lo_y, lo_z, L, unit} from the min/max words; returns true if
// a coordinate was not finite.
__device__ __forceinline__ bool box_from_minmax(const unsigned long long *mm, double *box)
{
    double ext = 0.0;
    for (int a = 0; a < 3; a++) {
        double lo = ord_to_dbl(mm[a]), hi = ord_to_dbl(mm[3 + a]);
        box[a] = lo;
        double e = __dsub_rn(hi, lo);
        ext = e > ext ? e : ext;
    }
    double L = 1.0;
    if (ext > 0.0) {
        while (L < ext) L *= 2.0;
        while (L / 2.0 >= ext) L /= 2.0;
    }
    box[3] = L;
    box[4] = L / 2097152.0;
    return mm[6] != 0ull;
}

__host__ __device__ __forceinline__ uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

// Inverse of spread3: the 21 bits at positions 0, 3, 6, ... packed together.
__host__ __device__ __forceinline__ int compact3(uint64_t x)
{
    x &= 0x1249249249249249ull;
    x = (x | x >> 2) & 0x10c30c30c30c30c3ull;
    x = (x | x >> 4) & 0x100f00f00f00f00full;
    x = (x | x >> 8) & 0x1f0000ff0000ffull;
    x = (x | x >> 16) & 0x1f00000000ffffull;
    x = (x | x >> 32) & 0x1fffffull;
    return (int)x;
}

// Exponent of the root box side L (a power of two).
__device__ __forceinline__ int box_lexp(double L)
{
    return (int)((__double_as_longlong(L) >> 52) & 0x7ff) - 1023;
}

// Morton grid cell of coordinate x: floor((x - lo) * 2^21 / L) clamped to
// [0, 2^21 - 1], L = 2^lexp, with x - lo the rounded FP64 difference.  The
// scale is a power of two, so the floor is read exactly from the bits of the
// difference with integer operations (GB300's FP64 pipe is narrow).  *res,
// when given, is the remainder x - lo - cell L / 2^21 (exact in FP64) in
// FP32, within one FP32 rounding.
__device__ __forceinline__ int grid_cell(double x, double lo, int lexp, float *res = nullptr)
{
    const double d = __dsub_rn(x, lo);  // >= 0
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    int e = (int)(b >> 52);
    unsigned long long m = b & 0xfffffffffffffull;
    if (e == 0) e = 1;  // subnormal
    else m |= 1ull << 52;
    const int s = 1054 + lexp - e;  // d = m 2^(e - 1075); one cell = 2^s units of m
    unsigned long long c = s >= 64 ? 0ull : (s <= 0 ? (unsigned long long)GNB_GRID_MAX : m >> s);
    if (c > GNB_GRID_MAX) c = GNB_GRID_MAX;
    if (res) {
        const unsigned long long f = s >= 64 ? m : (s <= 0 ? 0ull : m - (c << s));
        const float v = __uint2float_rn((unsigned)(f >> 32)) * 4294967296.f + __uint2float_rn((unsigned)f);
        *res = ldexpf(v, e - 1075);
    }
    return (int)c;
}

__device__ __forceinline__ uint64_t morton_key(int c0, int c1, int c2)
{
    return (spread3((uint32_t)c0) << 2) | (spread3((uint32_t)c1) << 1) | spread3((uint32_t)c2);
}

}  // namespace gnb
