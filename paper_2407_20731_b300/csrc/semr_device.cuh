// Device helpers shared by the reduce kernels: look-back state access,
// exact power-of-two scaling, magnitude thresholds, the even-odd folded 1-D
// transforms, FP32-pair ("df64") arithmetic, integer double->float
// conversion, exact fixed-point warp sums, and a warp sort and scan of
// 64-bit keys.
#pragma once

#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "semr_internal.h"

namespace semr {

// ------------------------------------------------------ bounds build
//
// Built with -DSEMR_BOUNDS, every kernel passes the index or byte-range test
// of each global access it makes to bchk() first: a test that fails sets
// SEMR_STATUS_BOUNDS and the caller skips the access (nothing traps).  In
// the default build bchk() is the constant true and the tests compile away.
#ifdef SEMR_BOUNDS
constexpr bool kBoundsBuild = true;
#else
constexpr bool kBoundsBuild = false;
#endif
__device__ __forceinline__ bool bchk(bool inside, unsigned* status) {
    if constexpr (kBoundsBuild) {
        if (!inside) atomicOr(status, static_cast<unsigned>(SEMR_STATUS_BOUNDS));
        return inside;
    }
    return true;
}

// ------------------------------------------------------ memory ordering

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Decoupled look-back, one warp: each round reads the states of the 32
// preceding tiles at once, adds the aggregates up to the nearest inclusive
// prefix, and stops there (predecessors before tile 0 count as a prefix of 0).
// Bounded: after 2^22 rounds that saw an unpublished tile it sets
// SEMR_STATUS_TIMEOUT and returns what it has.  Lane 0 publishes the tile's
// inclusive prefix.  Call with all 32 lanes.
__device__ __forceinline__ uint64_t lookback_warp(uint64_t* tile_state, uint64_t tile, uint64_t agg,
                                                  unsigned* status) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) return 0;  // tile 0 published its prefix with its aggregate
    uint64_t excl = 0;
    int64_t base = (int64_t)tile - 1;
    uint32_t spins = 0;
    while (true) {
        const int64_t j = base - lane;
        const uint64_t v = (j >= 0) ? ld_acquire_u64(&tile_state[j]) : kFlagPrefix;
        const uint64_t flag = v & ~kValueMask;
        const unsigned pmask = __ballot_sync(0xffffffffu, flag == kFlagPrefix);
        const unsigned xmask = __ballot_sync(0xffffffffu, flag == 0);
        const int first_p = pmask ? __ffs(pmask) - 1 : 32;
        const unsigned before = (first_p == 32) ? 0xffffffffu : ((1u << first_p) - 1u);
        if (xmask & before) {  // a nearer tile has not published yet: wait and reread
            if (++spins > (1u << 22)) {
                if (lane == 0) atomicOr(status, (unsigned)SEMR_STATUS_TIMEOUT);
                break;
            }
            __nanosleep(32);
            continue;
        }
        uint64_t c = (lane <= first_p) ? (v & kValueMask) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        excl += c;
        if (first_p < 32) break;
        base -= 32;
    }
    if (lane == 0) st_release_u64(&tile_state[tile], kFlagPrefix | ((excl + agg) & kValueMask));
    return excl;
}

// Decoupled look-back: exclusive prefix of tile `tile` given its aggregate.
// Bounded: after 2^22 polls it sets SEMR_STATUS_TIMEOUT and returns what it has.
__device__ __forceinline__ uint64_t lookback_exclusive(uint64_t* tile_state, uint64_t tile, uint64_t agg,
                                                       unsigned* status) {
    uint64_t excl = 0;
    if (tile == 0) return 0;
    int64_t j = (int64_t)tile - 1;
    uint32_t spins = 0;
    while (j >= 0) {
        const uint64_t v = ld_acquire_u64(&tile_state[j]);
        const uint64_t flag = v & ~kValueMask;
        if (flag == kFlagPrefix) {
            excl += v & kValueMask;
            break;
        } else if (flag == kFlagAggregate) {
            excl += v & kValueMask;
            --j;
        } else {
            if (++spins > (1u << 22)) {
                atomicOr(status, (unsigned)SEMR_STATUS_TIMEOUT);
                break;
            }
            __nanosleep(64);
        }
    }
    st_release_u64(&tile_state[tile], kFlagPrefix | ((excl + agg) & kValueMask));
    return excl;
}

// ------------------------------------------------------- exact scaling

__device__ __forceinline__ double pow2d(int e) {  // 2^e, e in [-1022, 1023]
    return __longlong_as_double((long long)(1023 + e) << 52);
}
__device__ __forceinline__ float pow2f(int e) {  // 2^e, e in [-126, 127]
    return __int_as_float((127 + e) << 23);
}

// Neighbours of a positive finite float/double by one unit in the last place.
__device__ __forceinline__ double next_up(double g) { return __longlong_as_double(__double_as_longlong(g) + 1); }
__device__ __forceinline__ double next_down(double g) { return __longlong_as_double(__double_as_longlong(g) - 1); }
__device__ __forceinline__ float next_upf(float g) { return __int_as_float(__float_as_int(g) + 1); }
__device__ __forceinline__ float next_downf(float g) { return __int_as_float(__float_as_int(g) - 1); }

// Smallest double g > 0 with fl(g*g) >= t (t normal, finite, > 0).  fl(g*g)
// is monotone in g, so |a| >= g  <=>  fl(a*a) >= t for every double a.
__device__ __forceinline__ double threshold_abs64(double t) {
    double g = sqrt(t);
    for (int it = 0; it < 4 && g * g < t; ++it) g = next_up(g);
    for (int it = 0; it < 4 && g > 0.0; ++it) {
        const double pr = next_down(g);
        if (pr * pr >= t) g = pr; else break;
    }
    return g;
}
// Smallest float g > 0 with (double)g * g >= t.  (double)g*g is exact, so
// |a| >= g  <=>  (double)a*a >= t  exactly, for every float a.
__device__ __forceinline__ float threshold_abs32(double t) {
    const double g64 = sqrt(t);
    if (g64 > (double)FLT_MAX) return __int_as_float(0x7f800000);  // +inf: nothing passes
    float g = (float)g64;
    if (g == 0.0f) g = __int_as_float(1);  // smallest subnormal
    for (int it = 0; it < 4 && (double)g * (double)g < t; ++it) g = next_upf(g);
    for (int it = 0; it < 4 && g > 0.0f; ++it) {
        const float pr = next_downf(g);
        if ((double)pr * (double)pr >= t) g = pr; else break;
    }
    return g;
}

// threshold_abs32 with a float square root as the first guess: the exact
// adjustment steps need only FP64 multiplies and compares (a float squared is
// exact in double), which keeps the FP64 latency per element short.
__device__ __forceinline__ float threshold_abs32_fast(double t) {
    if (t > 1.0e76) return threshold_abs32(t);  // outside the float range of the guess
    float g = sqrtf(__double2float_rn(t));
    if (!(g > 0.0f)) g = __int_as_float(1);
    for (int it = 0; it < 8 && (double)g * (double)g < t; ++it) g = next_upf(g);
    for (int it = 0; it < 8 && g > 0.0f; ++it) {
        const float pr = next_downf(g);
        if ((double)pr * (double)pr >= t) g = pr; else break;
    }
    return g;
}

// ------------------------------------------ double -> float without FP64 ops

// Round-toward-zero conversion of a double with |u| in the normal float
// range (or zero) using integer instructions only (B300 runs F2F on its
// slow FP64 pipe).  Magnitudes below 2^-126 come out as zero.
__device__ __forceinline__ float d2f_rz(double u) {
    const int lo = __double2loint(u), hi = __double2hiint(u);
    const int t = (hi & 0x7fffffff) - 0x38000000;  // rebias the exponent: 1023 -> 127
    const int f = t > 0 ? __funnelshift_l(lo, t, 3) : 0;  // (t << 3) | (lo >> 29)
    return __int_as_float(f | (hi & 0x80000000));
}
// d2f_rz of u 2^-ke, for an exact power-of-two prescale given as kb = ke << 20.
__device__ __forceinline__ float d2f_rz_scaled(double u, int kb) {
    const int lo = __double2loint(u), hi = __double2hiint(u);
    const int t = (hi & 0x7fffffff) - 0x38000000 - kb;
    const int f = t > 0 ? __funnelshift_l(lo, t, 3) : 0;
    return __int_as_float(f | (hi & 0x80000000));
}
// Prescale exponent of an element from its largest high word of |u| (sign
// cleared): ke with max |u| 2^-ke in [1, 2); 0 for an element of zeros and
// subnormals (hmax < 2^20), at most 1023.
__device__ __forceinline__ int prescale_exponent(uint32_t hmax) {
    return hmax < 0x00100000u ? 0 : min((int)(hmax >> 20) - 1023, 1023);
}
// Element flags from the same word: NaN, infinity or |u| >= 2^500 (energies
// beyond FP64); only subnormal values (|u| < 2^-1022).
__device__ __forceinline__ bool hmax_bad(uint32_t hmax) { return hmax >= ((uint32_t)(1023 + 500) << 20); }
__device__ __forceinline__ bool hmax_tiny(uint32_t hmax) { return hmax < 0x00100000u; }

// Split u 2^-ke into uh + ul, for an exact power-of-two prescale given as
// kb = ke << 20: uh = u 2^-ke rounded toward zero to 24 bits, ul the
// remaining 29 mantissa bits rounded to a float (so |u 2^-ke - uh - ul| <=
// 2^-48 |u 2^-ke|); both exactly 0 when |u 2^-ke| < 2^-126.  Integer
// instructions plus one I2F and one FMUL.
__device__ __forceinline__ void d2f_split(double u, int kb, float& uh, float& ul) {
    const int lo = __double2loint(u), hi = __double2hiint(u);
    const int e = ((hi >> 20) & 0x7ff) - (kb >> 20);
    const int t = (hi & 0x7fffffff) - 0x38000000 - kb;  // rebias the exponent: 1023 + ke -> 127
    uh = __int_as_float((t > 0 ? __funnelshift_l(lo, t, 3) : 0) | (hi & 0x80000000));
    // remainder: (lo & 0x1fffffff) * 2^(e - 1075)
    const float rem = __uint2float_rn((unsigned)lo & 0x1fffffffu);
    const int se = e - 1075;  // exponent of the remainder's unit
    // 2^se in two steps when it is below the normal float range (2^-64 is exact)
    const float r = (se >= -126) ? rem * pow2f(se)
                                 : (se >= -190 ? (rem * pow2f(se + 64)) * 5.421010862427522e-20f : 0.0f);
    ul = (t > 0) ? __int_as_float(__float_as_int(r) | (hi & 0x80000000)) : 0.0f;
}


// ------------------------------------------------- FP32-pair arithmetic

struct f2 {
    float h, l;
};
__device__ __forceinline__ f2 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ f2 df_add(f2 a, f2 b) {
    const f2 s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ f2 df_sub(f2 a, f2 b) { return df_add(a, {-b.h, -b.l}); }
__device__ __forceinline__ f2 df_mul(f2 a, f2 b) {
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.h, -p);
    return fast_two_sum(p, fmaf(a.h, b.l, fmaf(a.l, b.h, e)));
}
__device__ __forceinline__ f2 df_mulf(f2 a, float b) {  // a * b, b a float
    const float p = a.h * b;
    const float e = fmaf(a.h, b, -p);
    return fast_two_sum(p, fmaf(a.l, b, e));
}
// acc += a * b; the low word collects the rounding errors, renormalise with df_norm.
__device__ __forceinline__ void df_fma_acc(f2& acc, f2 a, f2 b) {
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)));
    const f2 s = two_sum(acc.h, p);
    acc.h = s.h;
    acc.l += s.l + e;
}
__device__ __forceinline__ f2 df_norm(f2 a) { return fast_two_sum(a.h, a.l); }
__device__ __forceinline__ f2 df_abs(f2 a) { return a.h < 0.0f ? f2{-a.h, -a.l} : a; }
// a >= b for normalised pairs
__device__ __forceinline__ bool df_ge(f2 a, f2 b) { return a.h > b.h || (a.h == b.h && a.l >= b.l); }
__device__ __forceinline__ f2 df_from_double(double g) {  // FP64 -> pair (once per element)
    const float h = (float)g;
    return {h, (float)(g - (double)h)};
}

// Double value of a normalised float pair, as its 64-bit pattern (one FP64
// add; used once per thread, not per point).
__device__ __forceinline__ unsigned long long pair_to_double_bits(f2 a) {
    return (unsigned long long)__double_as_longlong((double)a.h + (double)a.l);
}

// ------------------------------------------- exact fixed-point warp sums

// Value of a non-negative float x as the integer floor(x * 2^K), for
// x * 2^K < 2^61 (larger values saturate the caller's headroom check).
__device__ __forceinline__ unsigned long long fixp(float x, int K) {
    const unsigned b = __float_as_uint(x);
    const int ebits = (int)(b >> 23);
    if (ebits == 0) return 0ull;  // zero or subnormal: below any useful K
    const unsigned long long m = (b & 0x7fffffu) | 0x800000u;
    const int sh = ebits - 150 + K;  // x = m * 2^(ebits - 150)
    if (sh >= 0) return sh > 39 ? (1ull << 62) : (m << sh);
    return -sh > 31 ? 0ull : (m >> (-sh));
}
// Signed variant for the low word of a pair (|x| below the high word).
__device__ __forceinline__ long long fixp_signed(float x, int K) {
    const long long v = (long long)fixp(fabsf(x), K);
    return x < 0.0f ? -v : v;
}
// Exact sum over the warp of 62-bit non-negative integers: three 20-bit
// chunk sums with the warp reduction instruction.
__device__ __forceinline__ unsigned long long warp_sum_u62(unsigned long long v) {
    const unsigned c0 = (unsigned)(v & 0xfffffull), c1 = (unsigned)((v >> 20) & 0xfffffull),
                   c2 = (unsigned)(v >> 40);
    const unsigned long long s0 = __reduce_add_sync(0xffffffffu, c0);
    const unsigned long long s1 = __reduce_add_sync(0xffffffffu, c1);
    const unsigned long long s2 = __reduce_add_sync(0xffffffffu, c2);
    return s0 + (s1 << 20) + (s2 << 40);
}

// Ascending bitonic sort of one 64-bit key per lane across the warp.
__device__ __forceinline__ unsigned long long warp_sort_u64(unsigned long long v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, j);
            const bool up = (lane & k) == 0, low = (lane & j) == 0;  // block direction, lower lane of the pair
            v = (low == up) ? (v < o ? v : o) : (v < o ? o : v);
        }
    }
    return v;
}

// Inclusive prefix sum of one 64-bit value per lane (exact, lane order).
__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// ------------------------------------------------ 1-D folded transforms

// y_p = sum_i A[p][i] x_i using A[p][N-i] = (-1)^p A[p][i].
template <int LX, typename T>
__device__ __forceinline__ void fwd1d(const T* __restrict__ A, const T (&x)[LX], T (&y)[LX]) {
    constexpr int H = LX / 2;
    T ev[H > 0 ? H : 1], od[H > 0 ? H : 1];
#pragma unroll
    for (int i = 0; i < H; ++i) {
        ev[i] = x[i] + x[LX - 1 - i];
        od[i] = x[i] - x[LX - 1 - i];
    }
#pragma unroll
    for (int p = 0; p < LX; ++p) {
        T s;
        if ((p & 1) == 0) {
            if constexpr (LX & 1) {
                s = A[p * LX + H] * x[H];
#pragma unroll
                for (int i = 0; i < H; ++i) s = fma(A[p * LX + i], ev[i], s);
            } else {
                s = A[p * LX] * ev[0];
#pragma unroll
                for (int i = 1; i < H; ++i) s = fma(A[p * LX + i], ev[i], s);
            }
        } else {
            s = A[p * LX] * od[0];
#pragma unroll
            for (int i = 1; i < H; ++i) s = fma(A[p * LX + i], od[i], s);
        }
        y[p] = s;
    }
}

// y_i = sum_p Phi[i][p] x_p using Phi[N-i][p] = (-1)^p Phi[i][p].
template <int LX, typename T>
__device__ __forceinline__ void inv1d(const T* __restrict__ Phi, const T (&x)[LX], T (&y)[LX]) {
    constexpr int H = LX / 2;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        T e = Phi[i * LX] * x[0];
        T o = Phi[i * LX + 1] * x[1];
#pragma unroll
        for (int p = 2; p < LX; ++p) {
            if ((p & 1) == 0) e = fma(Phi[i * LX + p], x[p], e);
            else o = fma(Phi[i * LX + p], x[p], o);
        }
        y[i] = e + o;
        y[LX - 1 - i] = e - o;
    }
    if constexpr (LX & 1) {
        T e = Phi[H * LX] * x[0];
#pragma unroll
        for (int p = 2; p < LX; p += 2) e = fma(Phi[H * LX + p], x[p], e);
        y[H] = e;
    }
}

// FP32-pair versions: tables as (hi, lo) pairs.
template <int LX>
__device__ __forceinline__ void fwd1d_df(const float* __restrict__ Ah, const float* __restrict__ Al,
                                         const f2 (&x)[LX], f2 (&y)[LX]) {
    constexpr int H = LX / 2;
    f2 ev[H > 0 ? H : 1], od[H > 0 ? H : 1];
#pragma unroll
    for (int i = 0; i < H; ++i) {
        ev[i] = df_add(x[i], x[LX - 1 - i]);
        od[i] = df_sub(x[i], x[LX - 1 - i]);
    }
#pragma unroll
    for (int p = 0; p < LX; ++p) {
        f2 s = {0.0f, 0.0f};
        if ((p & 1) == 0) {
            if constexpr (LX & 1) df_fma_acc(s, {Ah[p * LX + H], Al[p * LX + H]}, x[H]);
#pragma unroll
            for (int i = 0; i < H; ++i) df_fma_acc(s, {Ah[p * LX + i], Al[p * LX + i]}, ev[i]);
        } else {
#pragma unroll
            for (int i = 0; i < H; ++i) df_fma_acc(s, {Ah[p * LX + i], Al[p * LX + i]}, od[i]);
        }
        y[p] = df_norm(s);
    }
}

template <int LX>
__device__ __forceinline__ void inv1d_df(const float* __restrict__ Ph, const float* __restrict__ Pl,
                                         const f2 (&x)[LX], f2 (&y)[LX]) {
    constexpr int H = LX / 2;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        f2 e = {0.0f, 0.0f}, o = {0.0f, 0.0f};
#pragma unroll
        for (int p = 0; p < LX; ++p) {
            if ((p & 1) == 0) df_fma_acc(e, {Ph[i * LX + p], Pl[i * LX + p]}, x[p]);
            else df_fma_acc(o, {Ph[i * LX + p], Pl[i * LX + p]}, x[p]);
        }
        e = df_norm(e);
        o = df_norm(o);
        y[i] = df_add(e, o);
        y[LX - 1 - i] = df_sub(e, o);
    }
    if constexpr (LX & 1) {
        f2 e = {0.0f, 0.0f};
#pragma unroll
        for (int p = 0; p < LX; p += 2) df_fma_acc(e, {Ph[H * LX + p], Pl[H * LX + p]}, x[p]);
        y[H] = df_norm(e);
    }
}

// ------------------------------------------------------ finalize

// Deterministic tree sum of a field's partials part[(f * nper + u) * 4 + {J e2,
// J E, Linf, max|u|}], u < nper: afterwards red[0..3][0] hold the two sums and
// the two maxima (256 threads; every thread passes the final barrier).
__device__ inline void finalize_tree(const double* part, int f, uint64_t nper, double (*red)[256]) {
    const int tid = threadIdx.x;
    double s0 = 0.0, s1 = 0.0, m2 = 0.0, m3 = 0.0;
    for (uint64_t u = tid; u < nper; u += 256) {
        const double* tp = part + 4 * ((uint64_t)f * nper + u);
        s0 += tp[0];
        s1 += tp[1];
        m2 = fmax(m2, tp[2]);
        m3 = fmax(m3, tp[3]);
    }
    red[0][tid] = s0;
    red[1][tid] = s1;
    red[2][tid] = m2;
    red[3][tid] = m3;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (tid < h) {
            red[0][tid] += red[0][tid + h];
            red[1][tid] += red[1][tid + h];
            red[2][tid] = fmax(red[2][tid], red[2][tid + h]);
            red[3][tid] = fmax(red[3][tid], red[3][tid + h]);
        }
        __syncthreads();
    }
}

// Field report of field f from its sums and maxima, the field's code count in
// the header (from the look-back states, p.tiles_per_field per field); field 0
// also writes the rest of the header and the summary.  One thread.
__device__ inline void finalize_report(const LaunchParams& p, int f, int lx, double se2, double sen, double linf,
                                       double umax) {
    // bounds build: the header, summary and state ranges follow from p alone, so field 0 (which
    // writes the summary's status) tests them for every field
    unsigned* status = &p.ctl->status;
    if (!bchk(f >= 0 && f < p.n_fields && p.n_fields <= SEMR_MAX_FIELDS && p.tiles_per_field >= 1 &&
                  kHeaderFixed + 8ull * p.n_fields <= p.header_bytes && p.header_bytes <= p.code_base &&
                  p.code_base <= p.payload_cap,
              status)) {
        if (f == 0) p.summary->status = *reinterpret_cast<volatile unsigned*>(status);
        return;
    }
    const uint64_t* tile_state = p.tile_state;
    const uint64_t n_tiles = (uint64_t)p.n_fields * p.tiles_per_field;
    const uint64_t t0 = (uint64_t)f * p.tiles_per_field;
    const uint64_t incl_end = tile_state[t0 + p.tiles_per_field - 1] & kValueMask;
    const uint64_t incl_beg = (f == 0) ? 0 : (tile_state[t0 - 1] & kValueMask);
    const uint64_t kept = incl_end - incl_beg;
    const uint64_t total = tile_state[n_tiles - 1] & kValueMask;
    semr_field_report* fr = &p.summary->field[f];
    fr->l2_abs = sqrt(se2);
    fr->l2_rel = sen > 0.0 ? sqrt(se2 / sen) : 0.0;
    fr->linf_abs = linf;
    fr->linf_rel = umax > 0.0 ? linf / umax : 0.0;
    fr->sum_err2 = se2;
    fr->sum_energy = sen;
    fr->umax = umax;
    fr->kept = kept;
    fr->bytes = p.fixed_bytes + (uint64_t)p.width * kept;
    const double orig = 8.0 * lx * lx * lx * (double)p.n_elem;
    fr->cr = 1.0 - (double)fr->bytes / orig;
    uint8_t* h = p.payload;
    *reinterpret_cast<uint64_t*>(h + kHeaderFixed + 8 * f) = kept;
    if (f == 0) {
        const uint64_t bytes = p.code_base + (uint64_t)p.width * total;
        h[0] = 'S'; h[1] = 'E'; h[2] = 'M'; h[3] = 'R';
        *reinterpret_cast<uint16_t*>(h + 4) = kPayloadVersion;
        *reinterpret_cast<uint16_t*>(h + 6) = (uint16_t)lx;
        *reinterpret_cast<uint16_t*>(h + 8) = (uint16_t)p.n_fields;
        uint16_t flags = 0;
        if (p.lossless) flags |= SEMR_PAYLOAD_LOSSLESS;
        if (p.width == 4) flags |= SEMR_PAYLOAD_CODE32;
        if (p.precision == SEMR_FP32) flags |= SEMR_PAYLOAD_FP32;
        if (p.cumulative) flags |= SEMR_PAYLOAD_CUMULATIVE;
        *reinterpret_cast<uint16_t*>(h + 10) = flags;
        *reinterpret_cast<uint32_t*>(h + 12) = (uint32_t)p.header_bytes;
        *reinterpret_cast<uint64_t*>(h + 16) = (uint64_t)p.n_elem;
        *reinterpret_cast<double*>(h + 24) = p.tau;
        *reinterpret_cast<uint64_t*>(h + 32) = p.code_base;
        *reinterpret_cast<uint64_t*>(h + 40) = total;
        for (uint64_t b = kHeaderFixed + 8ull * p.n_fields; b < p.header_bytes; ++b) h[b] = 0;
        p.summary->payload_bytes = bytes;
        p.summary->code_total = total;
        p.summary->n_fields = (uint32_t)p.n_fields;
        p.summary->cr = 1.0 - (double)bytes / (orig * p.n_fields);
        p.summary->status = p.ctl->status;
        p.summary->recomputed = p.ctl->recomputed;
    }
}


// Field f of one reduction: tree over its partials, then the report.  256 threads.
__device__ inline void finalize_field(const LaunchParams& p, int f, int lx, double (*red)[256], const double* part,
                                      uint64_t nper) {
    finalize_tree(part, f, nper, red);
    if (threadIdx.x == 0) finalize_report(p, f, lx, red[0][0], red[1][0], red[2][0], red[3][0]);
}

}  // namespace semr
