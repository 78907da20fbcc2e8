// Device helpers shared by the CUDA translation units: complex arithmetic on
// float2 / double2, small DFT butterflies and the Kaiser-Bessel polynomial.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hs {

template <typename R> struct CxT;
template <> struct CxT<float> { typedef float2 T; };
template <> struct CxT<double> { typedef double2 T; };
template <typename R> using Cx = typename CxT<R>::T;

template <typename R> __device__ __forceinline__ Cx<R> cx(R re, R im) {
    Cx<R> z;
    z.x = re;
    z.y = im;
    return z;
}
template <typename CT> __device__ __forceinline__ CT cadd(CT a, CT b) {
    a.x += b.x;
    a.y += b.y;
    return a;
}
template <typename CT> __device__ __forceinline__ CT csub(CT a, CT b) {
    a.x -= b.x;
    a.y -= b.y;
    return a;
}
template <typename CT> __device__ __forceinline__ CT cmul(CT a, CT b) {
    CT r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// a * conj(b)
template <typename CT> __device__ __forceinline__ CT cmulc(CT a, CT b) {
    CT r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}
template <typename CT, typename R> __device__ __forceinline__ CT cscale(CT a, R s) {
    a.x *= s;
    a.y *= s;
    return a;
}
// multiply by dir * i
template <int DIR, typename CT> __device__ __forceinline__ CT cmul_i(CT a) {
    CT r;
    r.x = -DIR * a.y;
    r.y = DIR * a.x;
    return r;
}

// 4-point DFT with kernel exp(DIR 2 pi i q r / 4), in place.
template <int DIR, typename CT> __device__ __forceinline__ void dft4(CT& a0, CT& a1, CT& a2, CT& a3) {
    CT s02 = cadd(a0, a2), d02 = csub(a0, a2);
    CT s13 = cadd(a1, a3), d13 = cmul_i<DIR>(csub(a1, a3));
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = cadd(d02, d13);
    a3 = csub(d02, d13);
}

// 8-point DFT with kernel exp(DIR 2 pi i q r / 8): split r = r1 + 4 r2, giving two
// 4-point DFTs on (a_r + a_{r+4}) and w^r (a_r - a_{r+4}), w = exp(DIR 2 pi i / 8);
// outputs interleave: X[2s] from the first, X[2s+1] from the second.
template <typename R, int DIR> __device__ __forceinline__ void dft8(Cx<R>* a) {
    typedef Cx<R> CT;
    const R h = (R)0.70710678118654752440;
    CT e0 = cadd(a[0], a[4]), e1 = cadd(a[1], a[5]), e2 = cadd(a[2], a[6]), e3 = cadd(a[3], a[7]);
    CT o0 = csub(a[0], a[4]), o1 = csub(a[1], a[5]), o2 = csub(a[2], a[6]), o3 = csub(a[3], a[7]);
    // w^1 = (1 + DIR i) / sqrt2, w^2 = DIR i, w^3 = (-1 + DIR i) / sqrt2
    o1 = cx<R>((o1.x - DIR * o1.y) * h, (o1.y + DIR * o1.x) * h);
    o2 = cmul_i<DIR>(o2);
    o3 = cx<R>((-o3.x - DIR * o3.y) * h, (-o3.y + DIR * o3.x) * h);
    dft4<DIR>(e0, e1, e2, e3);
    dft4<DIR>(o0, o1, o2, o3);
    a[0] = e0; a[2] = e1; a[4] = e2; a[6] = e3;
    a[1] = o0; a[3] = o1; a[5] = o2; a[7] = o3;
}

// Kaiser-Bessel piece evaluation: Horner in s = 2 f - 1.
template <typename R, int NC> __device__ __forceinline__ R horner(const R* c, R s) {
    R v = c[NC - 1];
#pragma unroll
    for (int k = NC - 2; k >= 0; --k) v = fma(v, s, c[k]);
    return v;
}

// x mod n for x in [-n, 2n): with m = n - 1 (n a power of two) the mask, with
// m < 0 (any other n) one conditional correction each way. m is uniform
// across a launch, so the choice never diverges.
__device__ __forceinline__ int wrapn(int x, int n, int m) {
    if (m >= 0) return x & m;
    x += x < 0 ? n : 0;
    return x >= n ? x - n : x;
}

// The wrap mask of wrapn for a period n.
__host__ __device__ __forceinline__ int wrap_mask(int n) { return (n & (n - 1)) == 0 ? n - 1 : -1; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of one double per thread (blockDim multiple of 32, <= 1024).
// Result valid in thread 0. `red` needs 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    __syncthreads();
    return v;
}

// Block-wide sum returned to every thread (uses red[0..32]).
__device__ __forceinline__ double block_sum_all(double v, double* red) {
    v = block_sum(v, red);
    if (threadIdx.x == 0) red[32] = v;
    __syncthreads();
    v = red[32];
    __syncthreads();
    return v;
}

}  // namespace hs
