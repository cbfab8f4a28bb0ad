// Device helpers of the warp-level reduce kernels (semr_warp.cu at lx = 8,
// semr_group.cu at the other orders): mbarrier waits with a bounded number of
// polls, the integer split of a double into a float pair with an exact
// power-of-two prescale, packed FP32x2 arithmetic (both pencils of a lane in
// one register pair), float-pair sums over a warp, the exact float threshold
// test, and a read-only look-back.
#pragma once

#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "semr_device.cuh"

namespace semr {

constexpr uint32_t kWaitPolls = 1000;      // bounded mbarrier polls, each suspending up to kWaitHintNs
constexpr uint32_t kWaitHintNs = 1000000;
constexpr unsigned FULL = 0xffffffffu;
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, %3;\n selp.u32 %0, 1, 0, P;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kWaitHintNs)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of bar (uniform over the warp): each poll sleeps until the
// phase completes or the hint elapses, so a waiting warp issues almost nothing.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    bool ok = false;
    for (uint32_t it = 0; it < kWaitPolls && !ok; ++it) ok = mbar_try_wait(bar, parity);
    return __all_sync(FULL, ok);
}
// Round-toward-zero float of u 2^-ke for a double u = (lo, hi), with bias = 0x38000000 + (ke << 20)
// (integer instructions; the exponent is rebiased from 1023 + ke to 127, so the scaling is exact;
// values with |u 2^-ke| < 2^-126 come out ~0).
__device__ __forceinline__ float w_d2f_rz(uint32_t lo, uint32_t hi, int bias) {
    const int t = max(static_cast<int>(hi & 0x7fffffffu) - bias, 0);
    return __uint_as_float(__funnelshift_l(lo, static_cast<uint32_t>(t), 3) | (hi & 0x80000000u));
}
// u 2^-ke = uh + ul: uh rounded toward zero to 24 bits, ul the next 23 bits (|u 2^-ke - uh - ul| <
// 2^-46 |u 2^-ke|); both zero-ish below 2^-80.
__device__ __forceinline__ void w_split(uint32_t lo, uint32_t hi, int bias, float& uh, float& ul) {
    uh = w_d2f_rz(lo, hi, bias);
    // mantissa bits 28..6 of the low word, an exact float integer via the 2^23 magic number
    const float m = __uint_as_float(((lo >> 6) & 0x7fffffu) | 0x4b000000u) - 8388608.0f;
    // their unit is 2^(E - 46) for uh = 1.x 2^E: exponent field of uh minus 46 (clamped at 0)
    const int ex = static_cast<int>(__float_as_uint(uh) & 0x7f800000u) - (46 << 23);
    ul = m * __uint_as_float(static_cast<uint32_t>(max(ex, 0)) | (hi & 0x80000000u));
}

// ---- packed FP32x2 arithmetic: the two pencils of a lane travel together as (s = 0, s = 1)
__device__ __forceinline__ float2 f2dup(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }

// Float pairs (hi + lo) of both pencils at once.
struct p2 {
    float2 h, l;
};
__device__ __forceinline__ p2 two_sum2(float2 a, float2 b) {
    const float2 s = f2add(a, b);
    const float2 bb = f2sub(s, a);
    return {s, f2add(f2sub(a, f2sub(s, bb)), f2sub(b, bb))};
}
__device__ __forceinline__ p2 fast_two_sum2(float2 a, float2 b) {
    const float2 s = f2add(a, b);
    return {s, f2sub(b, f2sub(s, a))};
}
__device__ __forceinline__ p2 df_norm2(p2 a) { return fast_two_sum2(a.h, a.l); }
__device__ __forceinline__ p2 df_sub2(p2 a, p2 b) {
    const p2 s = two_sum2(a.h, f2neg(b.h));
    return fast_two_sum2(s.h, f2add(s.l, f2sub(a.l, b.l)));
}
// acc += a * b; the low word collects the rounding errors (renormalise with df_norm2).
__device__ __forceinline__ void df_fma_acc2(p2& acc, p2 a, p2 b) {
    const float2 pr = f2mul(a.h, b.h);
    const float2 e = f2fma(a.h, b.l, f2fma(a.l, b.h, f2fma(a.h, b.h, f2neg(pr))));
    const p2 s = two_sum2(acc.h, pr);
    acc.h = s.h;
    acc.l = f2add(acc.l, f2add(s.l, e));
}

// Pair sum over the warp (butterfly: every lane ends with the same value).
__device__ __forceinline__ f2 warp_sum_pair(f2 s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = df_add(s, {__shfl_xor_sync(FULL, s.h, o), __shfl_xor_sync(FULL, s.l, o)});
    return s;
}
__device__ __forceinline__ float warp_sum_f(float s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    return s;
}
// Largest non-negative float over the warp (its bits order like unsigned integers).
__device__ __forceinline__ float warp_max_nonneg(float v) {
    return __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(v)));
}
// g^2 >= t exactly, for a float g and a normalised pair t.
__device__ __forceinline__ bool sq_ge(float g, f2 t) {
    const float ph = g * g;
    const float pl = fmaf(g, g, -ph);
    return ph > t.h || (ph == t.h && pl >= t.l);
}

// The second wait after a timed-out wait for a TMA block: the copy may still be in flight, and
// the CTA must not stop using its stage while it can land.  Waits once more (bounded, all 32
// lanes); if that wait gives up too, records SEMR_STATUS_STAGE: the copy may land after the
// kernel is done with the stage.  Returns whether the copy landed.
static __device__ __noinline__ bool drain_stage(uint64_t* bar, uint32_t parity, unsigned* status) {
    const bool ok = mbar_wait_bounded(bar, parity);
    if (!ok && (threadIdx.x & 31) == 0)
        atomicOr(status, static_cast<unsigned>(SEMR_STATUS_TIMEOUT | SEMR_STATUS_STAGE));
    return ok;
}

// Exclusive prefix of tile `tile` from its predecessors' states, as lookback_warp
// computes it, without publishing anything (bounded; all 32 lanes).
__device__ __forceinline__ uint64_t lookback_peek(const uint64_t* tile_state, uint64_t tile, unsigned* status) {
    const int lane = threadIdx.x & 31;
    uint64_t excl = 0;
    int64_t base = static_cast<int64_t>(tile) - 1;
    for (uint32_t spins = 0; base >= 0;) {
        const int64_t jj = base - lane;
        const uint64_t v = (jj >= 0) ? ld_acquire_u64(&tile_state[jj]) : kFlagPrefix;
        const uint64_t flag = v & ~kValueMask;
        const unsigned pmask = __ballot_sync(FULL, flag == kFlagPrefix);
        const unsigned xmask = __ballot_sync(FULL, flag == 0);
        const int first_p = pmask ? __ffs(pmask) - 1 : 32;
        const unsigned before = (first_p == 32) ? FULL : ((1u << first_p) - 1u);
        if (xmask & before) {
            if (++spins > (1u << 22)) {
                if (lane == 0) atomicOr(status, static_cast<unsigned>(SEMR_STATUS_TIMEOUT));
                break;
            }
            __nanosleep(64);
            continue;
        }
        uint64_t c = (lane <= first_p) ? (v & kValueMask) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
        excl += c;
        if (first_p < 32) break;
        base -= 32;
    }
    return excl;
}

// Finalize of field f by one warp of the CTA that finishes a single launch last (the CTA's
// warps take fields w, w + warps, ...): the sums and maxima over the field's tile partials in a
// fixed order (lane-strided sums, then a butterfly), then the exact maximum of |u| -- the kernel
// records each element's largest high word of |u|, which orders the elements like their
// maxima, so only the blocks whose high word is the field's are reread, each by the whole warp
// -- then the field report and (field 0) the header and summary.  A field whose every high
// word is 0 (zeros and subnormals) reports 0.  Every load is independent of the others, so the
// warp keeps many in flight.
__device__ inline void finalize_field_warp(const LaunchParams& p, int f, int lx, int tile) {
    const int lane = threadIdx.x & 31;
    const uint64_t nper = static_cast<uint64_t>(p.tiles_per_field);
    const uint64_t n3 = static_cast<uint64_t>(lx) * lx * lx;
    const double* tp = p.tile_part + 4 * (static_cast<uint64_t>(f) * nper);
    double s0 = 0.0, s1 = 0.0, m2 = 0.0, m3 = 0.0;
#pragma unroll 4
    for (uint64_t u = lane; u < nper; u += 32) {
        const double2 a = *reinterpret_cast<const double2*>(tp + 4 * u);
        const double2 b = *reinterpret_cast<const double2*>(tp + 4 * u + 2);
        s0 += a.x;
        s1 += a.y;
        m2 = fmax(m2, b.x);
        m3 = fmax(m3, b.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(FULL, s0, o);
        s1 += __shfl_xor_sync(FULL, s1, o);
        m2 = fmax(m2, __shfl_xor_sync(FULL, m2, o));
        m3 = fmax(m3, __shfl_xor_sync(FULL, m3, o));
    }
    const double M = m3;  // the field's largest high word, as a number
    const uint64_t E = static_cast<uint64_t>(p.n_elem);
    const uint32_t* um = p.hmax_elem + static_cast<uint64_t>(f) * E;
    const double* src = p.fields[f];
    unsigned long long umax = 0ull;
    for (uint64_t u0 = 0; M > 0.0 && u0 < nper; u0 += 32) {
        const uint64_t u = u0 + lane;
        for (unsigned tb = __ballot_sync(FULL, u < nper && tp[4 * u + 3] == M); tb; tb &= tb - 1) {
            const uint64_t t = u0 + (__ffs(tb) - 1);  // a tile that holds the maximum
            const uint64_t ee = min(E, (t + 1) * static_cast<uint64_t>(tile));
            for (uint64_t e0 = t * tile; e0 < ee; e0 += 32) {
                const uint64_t e = e0 + lane;
                for (unsigned eb = __ballot_sync(FULL, e < ee && static_cast<double>(um[e]) == M); eb; eb &= eb - 1) {
                    const double* blk = src + (e0 + (__ffs(eb) - 1)) * n3;  // reread by the warp
                    for (uint64_t i = lane; i < n3; i += 32)
                        umax = max(umax, static_cast<unsigned long long>(__double_as_longlong(blk[i])) &
                                             0x7fffffffffffffffull);
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) umax = max(umax, __shfl_xor_sync(FULL, umax, o));
    if (lane == 0) finalize_report(p, f, lx, s0, s1, m2, __longlong_as_double(static_cast<long long>(umax)));
}

// Whether this CTA is the last of the launch to finish (every thread gets the answer; call with
// every thread after the CTA's last global write).  The counter lives in the control block.
__device__ __forceinline__ bool last_cta_done(unsigned* done_ctas) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();  // this CTA's partials, states, codes and status before the count
        s_last = atomicAdd(done_ctas, 1u) == gridDim.x - 1;
        if (s_last) __threadfence();  // and the others' before the finalize reads them
    }
    __syncthreads();
    return s_last != 0;
}

// Packed pair sum a + b of both pencils.
__device__ __forceinline__ p2 df_add2(p2 a, p2 b) {
    const p2 s = two_sum2(a.h, b.h);
    return fast_two_sum2(s.h, f2add(s.l, f2add(a.l, b.l)));
}


}  // namespace semr
