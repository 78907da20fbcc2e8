// Gram matrix S = Z Z^T of the L x N channel-major matrix Z = X (+ Xa) on the
// fifth-generation tensor cores (tcgen05, BF16 operands, FP32 accumulation in
// tensor memory): the one dense contraction of the nuclear-norm prox
// (Eq. "prox-L*", Algorithm 2 step 5), FP32 plans.
//
// Exact-digit scheme. The tensor cores' FP32 accumulation does not round to
// nearest, so products of arbitrary TF32 / BF16 numbers carry a bias of about
// one unit in the last place per MMA. Here every operand is a small integer
// and every partial sum an integer below 2^24, so nothing is ever rounded
// inside the tensor cores:
//   * per chunk of 64 pixels and channel i, e_i is the smallest integer with
//     |z_in| < 2^e_i over the chunk, and Q_in = rint(z_in 2^(23 - e_i)) is a
//     24-bit integer (quantisation error <= 2^-24 of 2^e_i, unbiased);
//   * Q = 2^16 a + 2^8 b + c with balanced digits |a|, |b|, |c| <= 128, each
//     exact in BF16; digit products are below 2^14 and their sums over a
//     chunk below 2^20;
//   * one MMA chain (M = 128: rows [a; b], N = 192: rows [a; b; c], K = 64
//     pixels in four K = 16 steps) yields aa, ab, ac (lanes 0..63) and
//     ba, bb, bc (lanes 64..127) as exact integers;
//   * z_i . z_j = 2^(e_i + e_j - 30) (2^16 aa + 2^8 (ab + ba) + ac + bb + ca)
//     up to terms below 2^-24 of the leading one (bc, cb, cc are dropped);
//     with Y = 2^16 aa + 2^8 ab + 2 ac (lane i) and W = 2^8 ba + bb (lane
//     64 + i), that is 2^(e_i + e_j - 31) (Y + Y^T + W + W^T), so every
//     accumulator lane needs one value per column.
// The scaled Y, W of every chunk are added into FP32 registers (round to
// nearest) and, every GT_FLUSH chunks, into (hi, lo) pairs in shared memory
// with the error-free two-sum (Knuth), so the sum over chunks is as exact as
// in FP64. Each CTA writes its upper-triangle partial S in FP64 for the
// fixed-order reduction across CTAs. Range: |z| < 2^60 (beyond it the FP32
// Gram overflows anyway); a larger value raises the plan's error flag (bit 2).
//
// Data path per CTA (one per SM, a contiguous range of 64-pixel chunks):
// cp.async streams the raw X (and Xa) rows GT_STAGES - 1 chunks ahead into
// shared memory (16-byte copies, rows padded to 272 bytes against bank
// conflicts); four threads per channel form z = x + xa, the chunk exponent
// and the digits, stored in the 128-byte-swizzled K-major operand layout; one
// thread issues the chunk's four MMAs into one of two accumulator buffers and
// commits them to the buffer's mbarrier (which also guards reuse of the
// operand buffer); while the tensor cores work on chunk i, all eight warps
// drain chunk i - 1 (warp w reads lanes 32 (w % 4) .. + 31, columns
// 32 (w / 4) .. + 31 of each block). Every mbarrier wait is bounded in time:
// on expiry the kernel raises the plan's error flag (bit 1), stops issuing
// work, waits for its copies and frees its tensor memory.
#include <algorithm>
#include <cstdint>

#include "hs_device.cuh"
#include "hs_internal.h"

#include <cuda_bf16.h>

namespace hs {

constexpr int GT_THREADS = 256;
constexpr int GT_CHUNK = 64;                    // pixels per chunk (one 128-byte BF16 operand row)
constexpr int GT_STAGES = 3;                    // raw chunks staged (two in flight ahead)
constexpr int GT_FLUSH = 16;                    // chunks added in registers between two-sum flushes
constexpr int GT_RAW_LD = 68;                   // raw row stride (floats): 64 + 4 padding
constexpr int GT_RAW_FLOATS = 2 * 64 * GT_RAW_LD;
constexpr int GT_OPND_BYTES = 192 * 128;        // rows a (0-63), b (64-127), c (128-191), 128 B each
constexpr int GT_LDA = 65;                      // accumulator row stride (floats; conflict-free columns)
constexpr int GT_TMEM_COLS = 512;               // two accumulator buffers of 192 columns (at 0, 256)
constexpr int GT_EMIN = -45, GT_EMAX = 60;      // chunk exponent range kept by the FP32 scales
constexpr size_t GT_SMEM = 1024 + 2 * GT_OPND_BYTES + (size_t)GT_STAGES * GT_RAW_FLOATS * 4 +
                           2 * 128 * GT_LDA * 4 + 2 * 64 * 4 + 32;
constexpr unsigned long long GT_WAIT_NS = 1000000000ull;   // bound of one mbarrier wait

// Instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1),
// A and B BF16 (bits 7-9, 10-12 = 1), both K-major, N = 192 (bits 17-22 =
// N/8), M = 128 (bits 24-28 = M/16).
constexpr uint32_t GT_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((192u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1 (bits 46-47).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused by swizzled K-major layouts)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;             // SWIZZLE_128B
    return d;
}

// Byte offset of the 16-byte chunk c (0..7) of operand row r in the SW128 layout.
__device__ __forceinline__ uint32_t sw128_off(int r, int c) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the completion of the mbarrier phase of the given parity; false
// once GT_WAIT_NS has passed without it.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (!mbar_test(bar, parity))
        if (globaltimer() - t0 > GT_WAIT_NS) return false;
    return true;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(GT_IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes (thread t: lane
// 32 * (warp % 4) + t, register k: column col + k).
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

// Balanced base-256 digits of the 24-bit integer Q = rint(z 2^(23 - e)), as BF16.
__device__ __forceinline__ void digits(float z, float scale, float& a, float& b, float& c) {
    const float q = rintf(z * scale);
    a = rintf(q * (1.0f / 65536.0f));
    const float r = fmaf(-65536.0f, a, q);
    b = rintf(r * (1.0f / 256.0f));
    c = fmaf(-256.0f, b, r);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

__global__ void __launch_bounds__(GT_THREADS, 1)
    k_gram_tc(const float* __restrict__ X, const float* __restrict__ Xa, int L, int64_t N,
              double* __restrict__ part, int* __restrict__ err) {
    extern __shared__ uint8_t gt_smem[];
    uint8_t* base = (uint8_t*)(((uintptr_t)gt_smem + 1023) & ~(uintptr_t)1023);
    uint8_t* opnd = base;                                                 // 2 operand buffers
    float* raw = (float*)(base + 2 * GT_OPND_BYTES);                      // GT_STAGES raw chunks
    float* acc_hi = raw + GT_STAGES * GT_RAW_FLOATS;                      // 128 x GT_LDA
    float* acc_lo = acc_hi + 128 * GT_LDA;
    int* ex = (int*)(acc_lo + 128 * GT_LDA);                              // 2 x 64 chunk exponents
    uint64_t* mbar = (uint64_t*)(ex + 128);                               // 2 (8-byte aligned)
    uint32_t* tmem_slot = (uint32_t*)(mbar + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t nch_all = N / GT_CHUNK;
    const int64_t c_begin = nch_all * blockIdx.x / gridDim.x;
    const int nch = (int)(nch_all * (blockIdx.x + 1) / gridDim.x - c_begin);

    for (int i = tid; i < 2 * GT_OPND_BYTES / 16; i += GT_THREADS) ((uint4*)opnd)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < 2 * 128 * GT_LDA; i += GT_THREADS) acc_hi[i] = 0.f;
    for (int i = tid; i < 128; i += GT_THREADS) ex[i] = 0;
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(GT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int na = Xa ? 2 : 1;
    auto issue = [&](int i) {   // chunk i of this CTA into raw stage i % GT_STAGES
        if (i < nch) {
            const int64_t n0 = (c_begin + i) * GT_CHUNK;
            float* rs = raw + (i % GT_STAGES) * GT_RAW_FLOATS;
            for (int q = tid; q < na * L * 16; q += GT_THREADS) {
                const int a = q / (L * 16);
                const int rem = q - a * L * 16;
                const int l = rem >> 4, c = rem & 15;
                cp_async16(rs + (a * 64 + l) * GT_RAW_LD + 4 * c, (a ? Xa : X) + (int64_t)l * N + n0 + 4 * c);
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int d = 0; d < GT_STAGES - 1; ++d) issue(d);

    // Drain thread roles: accumulator lane r = 32 (warp % 4) + lane, columns
    // j0 .. j0 + 31 of each 64-column block. Lanes < 64 hold Y, the others W.
    const int r = 32 * (warp & 3) + lane;
    const int j0 = 32 * (warp >> 2);
    const bool yrow = r < 64;
    const int ei_row = r & 63;
    float acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k] = 0.f;

    // Convert-thread roles: channel cl = tid / 4 and pixels 16 (tid % 4) .. + 15.
    const int cl = tid >> 2, cq = tid & 3;

    int bad = 0, aborted = 0, range = 0;
    int issued_commits = 0;   // tid 0: commits made (for the bounded drain on abort)
    auto drain = [&](int i) {  // chunk i (committed on mbar[i & 1]) into the registers
        if (!__all_sync(0xffffffffu, mbar_wait(&mbar[i & 1], (i >> 1) & 1))) {
            bad = 1;
            return;
        }
        __syncwarp();
        tc_fence_after();
        const uint32_t t0 = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((i & 1) * 256 + j0);
        const int* exi = ex + (i & 1) * 64;
        const int e_r = exi[ei_row] - 31;
        float v[32], y[32];
        if (yrow) {
            tc_ld32(t0 + 128, v);                                       // ac
#pragma unroll
            for (int k = 0; k < 32; ++k) y[k] = 2.0f * v[k];
            tc_ld32(t0 + 64, v);                                        // ab
#pragma unroll
            for (int k = 0; k < 32; ++k) y[k] = fmaf(256.0f, v[k], y[k]);
            tc_ld32(t0, v);                                             // aa
#pragma unroll
            for (int k = 0; k < 32; ++k) y[k] = fmaf(65536.0f, v[k], y[k]);
        } else {
            tc_ld32(t0 + 64, v);                                        // bb
#pragma unroll
            for (int k = 0; k < 32; ++k) y[k] = v[k];
            tc_ld32(t0, v);                                             // ba
#pragma unroll
            for (int k = 0; k < 32; ++k) y[k] = fmaf(256.0f, v[k], y[k]);
        }
#pragma unroll
        for (int k = 0; k < 32; ++k) acc[k] = fmaf(pow2f(e_r + exi[j0 + k]), y[k], acc[k]);
        tc_fence_before();
    };
    auto flush = [&]() {       // registers -> (hi, lo) pairs, error-free
        float* hi = acc_hi + r * GT_LDA + j0;
        float* lo = acc_lo + r * GT_LDA + j0;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const float a = hi[k], sum = a + acc[k];
            const float bp = sum - a;
            lo[k] += (a - (sum - bp)) + (acc[k] - bp);
            hi[k] = sum;
            acc[k] = 0.f;
        }
    };

    for (int i = 0; i < nch; ++i) {
        issue(i + GT_STAGES - 1);
        cp_async_wait<GT_STAGES - 1>();
        if (__syncthreads_or(bad)) {          // chunk i staged by every thread
            aborted = 1;
            break;
        }
        const int s = i & 1;
        // operand buffer s was last read by the MMAs of chunk i - 2
        if (i >= 2 && !mbar_wait(&mbar[s], ((i - 2) >> 1) & 1)) bad = 1;
        {
            const float* rs = raw + (i % GT_STAGES) * GT_RAW_FLOATS;
            float z[16];
            float m = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float4 t = *(const float4*)(rs + cl * GT_RAW_LD + 16 * cq + 4 * k);
                if (Xa) {
                    const float4 u = *(const float4*)(rs + (64 + cl) * GT_RAW_LD + 16 * cq + 4 * k);
                    t.x += u.x;
                    t.y += u.y;
                    t.z += u.z;
                    t.w += u.w;
                }
                if (cl >= L) t = make_float4(0.f, 0.f, 0.f, 0.f);
                z[4 * k] = t.x;
                z[4 * k + 1] = t.y;
                z[4 * k + 2] = t.z;
                z[4 * k + 3] = t.w;
                m = fmaxf(m, fmaxf(fmaxf(fabsf(t.x), fabsf(t.y)), fmaxf(fabsf(t.z), fabsf(t.w))));
            }
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
            // smallest e with m < 2^e: the exponent of m plus one
            int e = ((__float_as_int(m) >> 23) & 0xFF) - 126;
            if (e > GT_EMAX) range = 1;
            e = min(max(e, GT_EMIN), GT_EMAX);
            if (cq == 0) ex[s * 64 + cl] = e;
            const float sc = pow2f(23 - e);
            uint32_t da[8], db[8], dc[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                float a0, b0, c0, a1, b1, c1;
                digits(z[2 * k], sc, a0, b0, c0);
                digits(z[2 * k + 1], sc, a1, b1, c1);
                da[k] = pack_bf16(a0, a1);
                db[k] = pack_bf16(b0, b1);
                dc[k] = pack_bf16(c0, c1);
            }
            if (cl < L) {
                uint8_t* op = opnd + s * GT_OPND_BYTES;
#pragma unroll
                for (int h = 0; h < 2; ++h) {   // 16-byte chunks 2 cq and 2 cq + 1 of the 128-byte row
                    const int c = 2 * cq + h;
                    *(uint4*)(op + sw128_off(cl, c)) = make_uint4(da[4 * h], da[4 * h + 1], da[4 * h + 2], da[4 * h + 3]);
                    *(uint4*)(op + sw128_off(64 + cl, c)) =
                        make_uint4(db[4 * h], db[4 * h + 1], db[4 * h + 2], db[4 * h + 3]);
                    *(uint4*)(op + sw128_off(128 + cl, c)) =
                        make_uint4(dc[4 * h], dc[4 * h + 1], dc[4 * h + 2], dc[4 * h + 3]);
                }
            }
        }
        fence_async_smem();
        tc_fence_before();
        if (__syncthreads_or(bad)) {          // operands of chunk i written
            aborted = 1;
            break;
        }
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(opnd + s * GT_OPND_BYTES);
            const uint32_t d_tmem = tmem + (uint32_t)(s * 256);
#pragma unroll
            for (int j = 0; j < 4; ++j) {     // K = 16 BF16 (32 bytes) per MMA
                const uint64_t d = sw128_desc(a0 + 32 * j);
                tc_mma_bf16(d_tmem, d, d, j == 0 ? 0u : 1u);
            }
            tc_commit(&mbar[s]);
            ++issued_commits;
        }
        if (i >= 1) {
            drain(i - 1);
            if ((i - 1) % GT_FLUSH == GT_FLUSH - 1) flush();
        }
    }
    if (!aborted && nch > 0) drain(nch - 1);
    flush();
    cp_async_wait<0>();
    if (__syncthreads_or(bad)) aborted = 1;   // the last drain may have expired
    if (__syncthreads_or(range) && tid == 0) atomicOr(err, 2);
    if (aborted && tid == 0) {
        atomicOr(err, 1);
        // let the last committed MMAs finish before the accumulators are freed (bounded)
        if (issued_commits > 0) {
            const int last = issued_commits - 1;
            (void)mbar_wait(&mbar[last & 1], (last >> 1) & 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (!aborted) {
        for (int q = tid; q < L * L; q += GT_THREADS) {
            const int i = q / L, j = q - i * L;
            if (i > j) continue;
            const auto v = [&](int row, int col) {
                return (double)acc_hi[row * GT_LDA + col] + (double)acc_lo[row * GT_LDA + col];
            };
            // the 2^-31 scale of the accumulated values already halves Y + Y^T + W + W^T
            const double sij = (v(i, j) + v(j, i)) + (v(64 + i, j) + v(64 + j, i));
            const int e_idx = i * L - i * (i - 1) / 2 + (j - i);   // row-major rank in the upper triangle
            part[(int64_t)e_idx * gridDim.x + blockIdx.x] = sij;
        }
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(GT_TMEM_COLS)
                     : "memory");
}

static int g_gram_tc_ctas = 0;

hs_status gram_tc_init() {
    int dev = 0, sms = 0;
    HS_CHECK_CUDA(cudaGetDevice(&dev));
    HS_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    HS_CHECK_CUDA(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GT_SMEM));
    g_gram_tc_ctas = sms;
    return HS_OK;
}

bool gram_tc_usable(const void* X, const void* Xa, int L, int64_t N) {
    const auto al = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
    return g_gram_tc_ctas > 0 && L >= 1 && L <= 64 && N % GT_CHUNK == 0 && al(X) && (Xa == nullptr || al(Xa));
}

// Partial Gram matrices of Z = X (+ Xa) into part[e * g + b] for the
// upper-triangle entry e and CTA b < g = *ctas_out (at most nparts CTAs).
hs_status gram_tc_launch(const float* X, const float* Xa, int L, int64_t N, double* part, int nparts, int* err,
                         int* ctas_out, cudaStream_t s) {
    const int64_t nch = N / GT_CHUNK;
    const int g = (int)std::min<int64_t>({(int64_t)g_gram_tc_ctas, (int64_t)nparts, std::max<int64_t>(nch, 1)});
    k_gram_tc<<<g, GT_THREADS, GT_SMEM, s>>>(X, Xa, L, N, part, err);
    HS_CHECK_LAUNCH();
    *ctas_out = g;
    return HS_OK;
}

}  // namespace hs
