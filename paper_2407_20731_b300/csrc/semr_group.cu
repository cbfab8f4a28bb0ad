// Warp-group fused reduce kernel for lx = 6 and lx = 10 (arXiv 2407.20731,
// Sec. IV-B: JPEG-like truncation of the modal Legendre coefficients of SEM
// element blocks, keeping the most energetic modes; Eq. 1 for the compression
// ratio).  The lx = 8 kernel (semr_warp.cu) maps an element's 64 pencils onto
// one warp exactly; 36 and 100 pencils do not divide that way, so here one
// element is reduced by a group of WPE warps (one at lx = 6, two at lx = 10):
//   * the element's contiguous block arrives in the group's stage by a 1-D
//     bulk copy (cp.async.bulk, mbarrier completion); its rows of 48 or 80
//     bytes are read by consecutive threads with conflict-free 16-byte loads;
//   * thread g of the group owns the pencils P = g and P = g + 32 WPE (the
//     second valid only while P < lx^2), packed as FP32x2 in every phase; the
//     forward transform contracts i in registers and j, k after two padded
//     transposes in the group's shared memory;
//   * the coefficients are then laid out once more, in mode order, so that
//     lane L of the group's warp w holds mode m = 32 k + L for the words k of
//     that warp: each ballot is exactly mask word k of the payload, and a
//     code's rank is a popcount prefix over the words, as at lx = 8;
//   * group sums are warp shuffles and, with two warps, one exchange through
//     shared memory behind a named barrier of the group's 64 threads;
//   * each group stages its codes in its own arena; the look-back tiles (32
//     elements per group), their one-tile-late resolution, the code placement
//     and the FP64 partials work as in the lx = 8 kernel.
// Precision modes as there: SEMR_FP32 runs FP32 transforms with an exact
// float-pair threshold test; SEMR_FP64 runs the forward transform in FP32
// under the proven error bound, recomputes in hardware FP64 every coefficient
// whose keep or rounding decision that bound cannot settle, and does the
// energy, reconstruction and error norms in float pairs.  Every element is
// read as u 2^-ke (an exact power-of-two prescale, ke the binary exponent of
// its largest |u|).  CUM selects the cumulative-energy truncation, as in the
// lx = 8 kernel, with the group's maxima and sums exchanged between its warps.
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>
#include <cstring>

#include "semr_device.cuh"
#include "semr_warp_common.cuh"

namespace semr {
namespace {

constexpr int GCTA = 128;  // threads per CTA (4 warps)

template <int LX>
struct GCfg {
    static constexpr int N3 = LX * LX * LX, NP = LX * LX;
    static constexpr int WPE = NP > 64 ? 2 : 1;          // warps per element group
    static constexpr int GT = 32 * WPE;                   // threads per group
    static constexpr int GPC = GCTA / GT;                 // groups per CTA
    static constexpr int TILE = 32 * GPC;                 // elements per look-back tile
    static constexpr int MW = (N3 + 31) / 32;             // mask words per element
    static constexpr int WPW = (MW + WPE - 1) / WPE;      // mask words per warp of the group
    static constexpr int MB = (N3 + 7) / 8;               // mask bytes per element in the payload
    static constexpr int LP = LX + 1;                     // transpose row stride (floats)
    static constexpr int PL = LX * LP;                    // transpose plane stride
    static constexpr int TB = LX * PL;                    // transpose buffer (floats)
    static_assert(2 * GT >= NP, "two pencils per thread cover the element");
    static_assert(TB >= 32 * MW, "the mode-ordered array fits the first transpose buffer");
    static_assert(TILE <= kWarpTile && TILE % 32 == 0, "tile bookkeeping of the lx = 8 layout");
};

template <bool DF>
__host__ __device__ constexpr int gsparse() { return DF ? 24 : 16; }  // kept-list capacity

template <int LX>
struct GTables {                 // as kernel parameters (constant bank)
    float2 A2[LX * LX];          // analysis A[p][i], duplicated for the packed transforms
    float Ph[LX * LX], Pl[LX * LX];  // synthesis Phi[i][p] (hi, lo)
    float wh[LX], wl[LX];        // GLL weights (hi, lo)
    float2 wh2[LX], wl2[LX];     // GLL weights duplicated (packed sums over a pencil)
    double A64[LX * LX];         // analysis A[p][i] in FP64 (the exact recomputation)
};

template <int LX>
struct GArgs {
    LaunchParams p;
    GTables<LX> tab;
    float tau_h, tau_l;
    uint32_t total_tiles;
};

struct GStash {    // one element's results, kept until the end of its tile
    int32_t ke;     // prescale exponent: the values below are those of u 2^-ke
    uint32_t hmax;  // largest high word of |u|
    float sh, sl;   // S = sum w u^2 (pair)
    float eh, el;   // e2 = sum w (u - u~)^2 (pair)
    float lh, ll;   // Linf = max |u - u~| (pair)
};
static_assert(sizeof(GStash) == 32, "stash entry");

template <int LX, bool DF, bool CUM = false>
struct GSmem {
    using C = GCfg<LX>;
    // per group
    static constexpr size_t stage = (8ull * C::N3 + 127) / 128 * 128;
    static constexpr size_t o_T = stage;                                  // 2 TB floats (one TB float2)
    static constexpr size_t o_bm = o_T + 8ull * C::TB;                    // MW mask words
    static constexpr size_t o_kl = o_bm + 4ull * ((C::MW + 3) / 4 * 4);   // kept list (mode, code)
    static constexpr size_t o_x = o_kl + 8ull * gsparse<DF>();            // exchange slots
    static constexpr size_t o_bar = o_x + 4ull * 32;
    static constexpr size_t o_ul = (o_bar + 8 + 15) / 16 * 16;            // parked words of u [LX][GT] float2
    static constexpr size_t o_uh = o_ul + 8ull * LX * C::GT;               // FP64 mode at lx = 10 with threshold
    static constexpr size_t gbytes =                                       // truncation: parked high words
        (o_uh + (DF && LX > 6 && !CUM ? 8ull * LX * C::GT : 0) + 127) / 128 * 128;
    // per CTA
    static constexpr size_t off_tab = C::GPC * gbytes;                    // Phi [i][p] and [p][i], hi and lo
    static constexpr size_t off_res = off_tab + 16ull * C::NP;            // GStash[TILE]
    static constexpr size_t bytes = off_res + sizeof(GStash) * C::TILE + 128;  // + alignment slack
};

// exchange slots of a group (floats/words): each written by warp w at [slot + w]
constexpr int XH = 0, XS = 2, XSL = 4, XC = 6, XE = 8, XEL = 10, XL = 12, XLL = 14, XA = 16;
// cumulative truncation (before XC..XLL are used for the element): the sums R, sum |a| and the count
// left, two alternating pairs for the per-extraction maxima, the smallest kept value; the general
// path's 64-bit sums use the words XC .. XC + 7 (two alternating pairs of two-word values)
constexpr int XR = 18, XB = 20, XN = 22, XM = 24, XV = 28;

template <int WPE>
__device__ __forceinline__ void gsync(int gi) {
    if constexpr (WPE == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + gi), "r"(32 * WPE) : "memory");
    }
}

// 1-D bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) into dst; completion on bar.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Folded forward transform of both pencils along one axis: y_p = sum_i A[p][i] x_i with
// A[p][LX-1-i] = (-1)^p A[p][i]; per output the product chain starts at A[p][0] and adds
// i = 1 .. H-1 in order (the order the host-side error-bound test replays).
template <int LX>
__device__ __forceinline__ void g_fwd2(const float2* __restrict__ A2, const float2 (&x)[LX], float2 (&y)[LX]) {
    constexpr int H = LX / 2;
    float2 ev[H], od[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
        ev[i] = f2add(x[i], x[LX - 1 - i]);
        od[i] = f2sub(x[i], x[LX - 1 - i]);
    }
#pragma unroll
    for (int p = 0; p < LX; ++p) {
        const float2* a = A2 + p * LX;
        float2 s = f2mul(a[0], (p & 1) ? od[0] : ev[0]);
#pragma unroll
        for (int i = 1; i < H; ++i) s = f2fma(a[i], (p & 1) ? od[i] : ev[i], s);
        y[p] = s;
    }
}

// Folded inverse in FP32 of both pencils: y_i = sum_p Phi[i][p] x_p with Phi[LX-1-i][p] = (-1)^p Phi[i][p].
template <int LX>
__device__ __forceinline__ void g_inv2(const float* __restrict__ Ph, const float2 (&x)[LX], float2 (&y)[LX]) {
    constexpr int H = LX / 2;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        float2 e = f2mul(f2dup(Ph[i * LX]), x[0]), o = f2mul(f2dup(Ph[i * LX + 1]), x[1]);
#pragma unroll
        for (int p = 2; p < LX; ++p) {
            if ((p & 1) == 0) e = f2fma(f2dup(Ph[i * LX + p]), x[p], e);
            else o = f2fma(f2dup(Ph[i * LX + p]), x[p], o);
        }
        y[i] = f2add(e, o);
        y[LX - 1 - i] = f2sub(e, o);
    }
}

// Folded inverse in float pairs of both pencils.
template <int LX>
__device__ __forceinline__ void g_inv_df2(const float* __restrict__ Ph, const float* __restrict__ Pl,
                                          const p2 (&x)[LX], p2 (&y)[LX]) {
    constexpr int H = LX / 2;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        p2 e = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)}, o = e;
#pragma unroll
        for (int p = 0; p < LX; ++p) {
            const p2 c = {f2dup(Ph[i * LX + p]), f2dup(Pl[i * LX + p])};
            if ((p & 1) == 0) df_fma_acc2(e, c, x[p]);
            else df_fma_acc2(o, c, x[p]);
        }
        e = df_norm2(e);
        o = df_norm2(o);
        y[i] = df_add2(e, o);
        y[LX - 1 - i] = df_sub2(e, o);
    }
}

// Exact coefficient a'[r][q][p] = 2^-ke sum A[r][k] A[q][j] A[p][i] u[k][j][i] of the element
// block at u (global memory) in hardware FP64, by one warp: lane L contracts the pencils (k, j) =
// L, L + 32, ... along i, then with A[q][j] A[r][k], and the warp sums.  FP64 because the
// decisions sent here can lie within ~1e-8 relative of a tie (small kept coefficients at small
// tau); rare, so the slow FP64 pipe costs little; the block is reread from L2.
template <int LX>
__device__ __noinline__ double g_exact_coef(const double* __restrict__ u, int pp, int qq, int rr,
                                            const double* __restrict__ A64, double sc) {
    constexpr int NP = LX * LX;
    const int lane = threadIdx.x & 31;
    double c = 0.0;
    for (int P = lane; P < NP; P += 32) {
        const int j = P % LX, k = P / LX;
        const double2* row = reinterpret_cast<const double2*>(u + P * LX);
        double xs = 0.0;
#pragma unroll
        for (int c2 = 0; c2 < LX / 2; ++c2) {
            const double2 v = __ldg(row + c2);
            xs = fma(A64[pp * LX + 2 * c2], v.x, xs);
            xs = fma(A64[pp * LX + 2 * c2 + 1], v.y, xs);
        }
        c = fma(xs * A64[qq * LX + j], A64[rr * LX + k], c);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    return c * sc;
}

// Settles the ambiguous decisions of this warp's modes (bit kk of amb: mode 32 (w0 + kk) + lane,
// value M[32 (w0 + kk) + lane]) exactly, one at a time over the warp; a kept one becomes its
// code times 2^s' (exact).  Returns the lane's updated keep bits.
template <int LX>
__device__ __noinline__ uint32_t g_resolve(float* M, int w0, uint32_t amb, uint32_t kb, const double* __restrict__ u,
                                           const double* __restrict__ A64, double sc, f2 t, float qd, float qu,
                                           unsigned& recomputed) {
    constexpr int NP = LX * LX;
    const int lane = threadIdx.x & 31;
    const double td = static_cast<double>(t.h) + static_cast<double>(t.l);
    while (__any_sync(FULL, amb != 0u)) {
        const int src = __ffs(__ballot_sync(FULL, amb != 0u)) - 1;
        const int kk = __shfl_sync(FULL, __ffs(amb) - 1, src);
        const int m = 32 * (w0 + kk) + src;
        const int pp = m % LX, qq = (m / LX) % LX, rr = m / NP;
        const double c = g_exact_coef<LX>(u, pp, qq, rr, A64, sc);
        ++recomputed;
        if (lane == src) {
            const bool keep = c * c >= td;
            float v = static_cast<float>(c);
            if (keep) v = static_cast<float>(rint(c * static_cast<double>(qd))) * qu;  // ties to even; exact
            M[m] = v;
            kb = keep ? (kb | (1u << kk)) : (kb & ~(1u << kk));
            amb &= ~(1u << kk);
        }
    }
    __syncwarp();
    return kb;
}

// Settles the rounding of this warp's kept modes of word w0 + kk that the FP32 bound leaves
// undecided (bit set in flag: mode 32 (w0 + kk) + lane), one at a time over the warp: each
// becomes its code times 2^s' (exact), also in M.  Returns the lane's value.
template <int LX>
__device__ __noinline__ float g_settle(float a, bool flag, float* M, int w0, int kk, const double* __restrict__ u,
                                       const double* __restrict__ A64, double sc, float qd, float qu,
                                       unsigned& recomputed) {
    constexpr int NP = LX * LX;
    const int lane = threadIdx.x & 31;
    for (uint32_t fl = __ballot_sync(FULL, flag); fl; fl &= fl - 1) {
        const int src = __ffs(fl) - 1;
        const int m = 32 * (w0 + kk) + src;
        const double c = g_exact_coef<LX>(u, m % LX, (m / LX) % LX, m / NP, A64, sc);
        ++recomputed;
        if (lane == src) {
            a = static_cast<float>(rint(c * static_cast<double>(qd))) * qu;  // ties to even; exact
            M[m] = a;
        }
    }
    __syncwarp();
    return a;
}

// Sum over the group of a per-warp value (both warps of an lx = 10 group call it; slot pair XS..
// in the exchange words, alternating by `parity` so that one barrier per call suffices).
template <int WPE>
__device__ __forceinline__ unsigned long long group_sum_u62(unsigned long long v, uint32_t* xu, int wg, int gi,
                                                           int parity) {
    v = warp_sum_u62(v);
    if constexpr (WPE == 1) {
        return v;
    } else {
        uint32_t* slot = xu + XC + 4 * parity;
        if ((threadIdx.x & 31) == 0) {
            slot[2 * wg] = static_cast<uint32_t>(v);
            slot[2 * wg + 1] = static_cast<uint32_t>(v >> 32);
        }
        gsync<WPE>(gi);
        return (static_cast<unsigned long long>(slot[1]) << 32 | slot[0]) +
               (static_cast<unsigned long long>(slot[3]) << 32 | slot[2]);
    }
}

// Cumulative-energy selection of an element that the fast path leaves open (a rare path, out
// of line; every thread of the group calls it): FP64 mode recomputes the element's coefficients
// 2^-ke A x A x A u in hardware FP64 from its doubles (reread from L2) through the group's buffer
// D (the transpose buffers, as doubles), the FP32 form takes its FP32 coefficients am as they
// are.  Energies become 64-bit fixed-point keys floor(a^2 2^K), t 2^K in [2^47, 2^48) (exact
// integer sums in any order), and a bisection on the key value finds T, the smallest key whose
// sum of keys up to it exceeds floor(t 2^K).  Returns the lane's keep bits (bit kk: mode
// 32 (w0 + kk) + lane); FP64 mode also rewrites the group's mode-ordered values M: each kept
// mode its code times 2^s' (exact), every other mode its value rounded to float.
template <int LX, int WPE, bool DF>
__device__ __noinline__ uint32_t g_cum_general(float* M, const float* am, uint32_t vm, int w0, int wg, int gi, int g,
                                               int P0, int P1, bool v1, uint32_t* xu,
                                               const double* __restrict__ u, const double* __restrict__ A64,
                                               double sc, double td, float qd, float qu, unsigned& recomputed) {
    constexpr int N3 = LX * LX * LX, NP = LX * LX, MW = (N3 + 31) / 32, WPW = (MW + WPE - 1) / WPE;
    const int lane = threadIdx.x & 31;
    double a64[WPW];
    if constexpr (DF) {
        double* D = reinterpret_cast<double*>(M);  // N3 doubles (the transpose buffers)
        double y[2][LX];
        gsync<WPE>(gi);  // every read of M as floats is done
#pragma unroll
        for (int s = 0; s < 2; ++s) {  // along i: pencils (k, j) -> D[k][j][p]
            const int P = s ? P1 : P0;
            if (s == 0 || v1) {
                const double* row = u + static_cast<size_t>(P) * LX;
                double x[LX];
#pragma unroll
                for (int i = 0; i < LX; ++i) x[i] = __ldg(row + i) * sc;
#pragma unroll
                for (int pp = 0; pp < LX; ++pp) {
                    double acc = 0.0;
#pragma unroll
                    for (int i = 0; i < LX; ++i) acc = fma(A64[pp * LX + i], x[i], acc);
                    y[s][pp] = acc;
                }
            }
        }
#pragma unroll
        for (int s = 0; s < 2; ++s)
            if (s == 0 || v1)
#pragma unroll
                for (int pp = 0; pp < LX; ++pp) D[(s ? P1 : P0) * LX + pp] = y[s][pp];
        gsync<WPE>(gi);
#pragma unroll
        for (int s = 0; s < 2; ++s) {  // along j: pencils (k, p) -> D[k][q][p]
            const int P = s ? P1 : P0;
            if (s == 0 || v1) {
                const int k = P / LX, pp = P % LX;
                double x[LX];
#pragma unroll
                for (int jj = 0; jj < LX; ++jj) x[jj] = D[(k * LX + jj) * LX + pp];
#pragma unroll
                for (int q = 0; q < LX; ++q) {
                    double acc = 0.0;
#pragma unroll
                    for (int jj = 0; jj < LX; ++jj) acc = fma(A64[q * LX + jj], x[jj], acc);
                    y[s][q] = acc;
                }
            }
        }
        gsync<WPE>(gi);
#pragma unroll
        for (int s = 0; s < 2; ++s)
            if (s == 0 || v1) {
                const int P = s ? P1 : P0, k = P / LX, pp = P % LX;
#pragma unroll
                for (int q = 0; q < LX; ++q) D[(k * LX + q) * LX + pp] = y[s][q];
            }
        gsync<WPE>(gi);
#pragma unroll
        for (int s = 0; s < 2; ++s) {  // along k: pencils (q, p) -> coefficient r, mode P + NP r
            const int P = s ? P1 : P0;
            if (s == 0 || v1) {
                const int q = P / LX, pp = P % LX;
                double x[LX];
#pragma unroll
                for (int kk = 0; kk < LX; ++kk) x[kk] = D[(kk * LX + q) * LX + pp];
#pragma unroll
                for (int r = 0; r < LX; ++r) {
                    double acc = 0.0;
#pragma unroll
                    for (int kk = 0; kk < LX; ++kk) acc = fma(A64[r * LX + kk], x[kk], acc);
                    y[s][r] = acc;
                }
            }
        }
        gsync<WPE>(gi);
#pragma unroll
        for (int s = 0; s < 2; ++s)
            if (s == 0 || v1)
#pragma unroll
                for (int r = 0; r < LX; ++r) D[(s ? P1 : P0) + NP * r] = y[s][r];
        gsync<WPE>(gi);
#pragma unroll
        for (int kk = 0; kk < WPW; ++kk) a64[kk] = ((vm >> kk) & 1u) ? D[32 * (w0 + kk) + lane] : 0.0;
        gsync<WPE>(gi);  // every double is read before M is rewritten as floats
        if (wg == 0) recomputed += N3;  // (counted once per element)
    } else {
#pragma unroll
        for (int kk = 0; kk < WPW; ++kk) a64[kk] = ((vm >> kk) & 1u) ? static_cast<double>(am[kk]) : 0.0;
    }
    int ex;
    frexp(td, &ex);  // td in [2^(ex - 1), 2^ex)
    const double sK = ldexp(1.0, 48 - ex);
    const unsigned long long tt = static_cast<unsigned long long>(td * sK);
    constexpr unsigned long long kClamp = 1ull << 50;
    unsigned long long key[WPW];
    unsigned long long own = 0ull;
#pragma unroll
    for (int kk = 0; kk < WPW; ++kk) {
        const double v = a64[kk] * a64[kk] * sK;
        key[kk] = v >= static_cast<double>(kClamp) ? kClamp : static_cast<unsigned long long>(v);
        own += key[kk];
    }
    int par = 0;
    uint32_t kb = 0;
    if (group_sum_u62<WPE>(own, xu, wg, gi, par) > tt) {  // else every energy fits the budget
        unsigned long long lo = 1, hi = kClamp;  // smallest v with sum_{key <= v} key > tt
        while (lo < hi) {
            const unsigned long long mid = lo + (hi - lo) / 2;
            unsigned long long sm = 0ull;
#pragma unroll
            for (int kk = 0; kk < WPW; ++kk) sm += key[kk] <= mid ? key[kk] : 0ull;
            par ^= 1;
            if (group_sum_u62<WPE>(sm, xu, wg, gi, par) > tt) hi = mid;
            else lo = mid + 1;
        }
#pragma unroll
        for (int kk = 0; kk < WPW; ++kk) kb |= (key[kk] >= lo ? 1u : 0u) << kk;
    }
    kb &= vm;
    if constexpr (DF) {
#pragma unroll
        for (int kk = 0; kk < WPW; ++kk)
            if ((vm >> kk) & 1u)
                M[32 * (w0 + kk) + lane] = ((kb >> kk) & 1u)
                                               ? static_cast<float>(rint(a64[kk] * static_cast<double>(qd))) * qu
                                               : static_cast<float>(a64[kk]);
    }
    gsync<WPE>(gi);  // (M complete; the exchange words are free again)
    (void)g;
    return kb;
}

template <int LX, int MODE, bool CUM>
struct GOcc {  // CTAs per SM the register budget aims at (measured)
    static constexpr int value = LX <= 6 ? (MODE ? (CUM ? 4 : 3) : 5) : 3;
};

// BATCH = false: one reduction, parameters in A.p.  BATCH = true: the work queue q of
// several reductions of this lx (each with its own descriptor, payload and scratch; they
// share one code staging).
template <int LX, int MODE, bool BATCH, bool CUM = false>
__global__ void __launch_bounds__(GCTA, GOcc<LX, MODE, CUM>::value)
    reduce_group_kernel(const __grid_constant__ GArgs<LX> A, const BatchQueue q) {
    using C = GCfg<LX>;
    constexpr bool DF = MODE != 0;
    using SM = GSmem<LX, DF, CUM>;
    constexpr int N3 = C::N3, NP = C::NP, GT = C::GT, GPC = C::GPC, WPE = C::WPE, TILE = C::TILE;
    constexpr int MW = C::MW, WPW = C::WPW, MB = C::MB, LP = C::LP, PL = C::PL, TB = C::TB;
    constexpr int KL = gsparse<DF>();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gi = threadIdx.x / GT, g = threadIdx.x % GT, wg = g >> 5;  // group, thread in group, warp in group

    // CTA tables: Phi [i][p] (hi, lo) and [p][i] (hi, lo)
    float* sPh = reinterpret_cast<float*>(smem + SM::off_tab);
    float* sPl = sPh + NP;
    float* sPTh = sPl + NP;
    float* sPTl = sPTh + NP;
    for (int t = threadIdx.x; t < NP; t += GCTA) {
        const int i = t / LX, c = t % LX;  // Ph[t] = Phi[i][c]
        sPh[t] = A.tab.Ph[t];
        sPl[t] = A.tab.Pl[t];
        sPTh[c * LX + i] = A.tab.Ph[t];
        sPTl[c * LX + i] = A.tab.Pl[t];
    }
    GStash* s_res = reinterpret_cast<GStash*>(smem + SM::off_res);
    uint8_t* gsm = smem + gi * SM::gbytes;
    uint8_t* stage = gsm;
    float* T = reinterpret_cast<float*>(gsm + SM::o_T);    // two TB-float buffers, or one of TB float2
    float* T2 = T + TB;
    float* M = T;                                            // mode-ordered values (aliases the first buffer)
    uint32_t* bm = reinterpret_cast<uint32_t*>(gsm + SM::o_bm);
    int2* skl = reinterpret_cast<int2*>(gsm + SM::o_kl);
    float* xf = reinterpret_cast<float*>(gsm + SM::o_x);
    uint32_t* xu = reinterpret_cast<uint32_t*>(gsm + SM::o_x);
    uint64_t* bar = reinterpret_cast<uint64_t*>(gsm + SM::o_bar);
    if (g == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    // this thread's pencils: P = g (slot 0) and P = g + GT (slot 1, valid while < NP)
    const int P0 = g, P1 = g + GT;
    const bool v1 = P1 < NP;
    const int k0 = P0 / LX, j0 = P0 % LX, k1 = v1 ? P1 / LX : 0, j1 = v1 ? P1 % LX : 0;
    // w_j w_k of the two nodal pencils (pairs), for the weighted sums over a pencil
    const f2 wjk0 = df_mul({A.tab.wh[j0], A.tab.wl[j0]}, {A.tab.wh[k0], A.tab.wl[k0]});
    const f2 wjk1 = v1 ? df_mul({A.tab.wh[j1], A.tab.wl[j1]}, {A.tab.wh[k1], A.tab.wl[k1]}) : f2{0.0f, 0.0f};

    const uint32_t total_tiles = BATCH ? static_cast<uint32_t>(q.total_tiles) : A.total_tiles;
    unsigned* counter = BATCH ? q.counter : &A.p.ctl->tile_counter;
    uint8_t* stage_cta = reinterpret_cast<uint8_t*>(BATCH ? q.items[0].code_stage : A.p.code_stage) +
                         static_cast<uint64_t>(blockIdx.x) * kWarpStageBytes;
    if (!bchk(static_cast<int>(blockIdx.x) < (BATCH ? q.items[0].stage_ctas : A.p.stage_ctas),
              BATCH ? &q.items[0].ctl->status : &A.p.ctl->status))
        return;  // (before any barrier or copy) a grid larger than the code staging
    int16_t* stage_codes = reinterpret_cast<int16_t*>(stage_cta);
    uint32_t* stage_pre = reinterpret_cast<uint32_t*>(stage_cta + 2ull * kWarpCtaWarps * kWarpArena * 2);
    uint32_t* stage_off = stage_pre + 2 * (kWarpTile + 1);
    constexpr uint32_t kDirect = 0xffffffffu;
    constexpr int ARENA = WPE * kWarpArena;  // the group's codes per tile parity

    __shared__ uint32_t s_tile[2];
    __shared__ uint32_t s_titem[2], s_tloc[2];    // their item and tile index within the item (BATCH)
    __shared__ LaunchParams s_par[BATCH ? 2 : 1];  // BATCH: descriptors of the current and previous tile
    auto resolve = [&](uint32_t gt, int slot) {    // item and local tile of a claimed tile (one thread)
        uint32_t item = 0, loc = gt;
        if (BATCH && gt < total_tiles) {           // last item whose first tile is <= gt
            int lo = 0, hi = q.n_items - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) / 2;
                if (q.tile_base[mid] <= gt) lo = mid; else hi = mid - 1;
            }
            item = static_cast<uint32_t>(lo);
            loc = gt - static_cast<uint32_t>(q.tile_base[lo]);
        }
        s_titem[slot] = item;
        s_tloc[slot] = loc;
    };
    __shared__ uint32_t s_cnt[TILE];  // tile tag << 16 | code count
    __shared__ unsigned long long s_excl;
    __shared__ unsigned long long s_peek;
    __shared__ uint32_t s_peek_tag;
    __shared__ double s_wpart[4][4];
    __shared__ int s_abort;
    if (threadIdx.x == 0) {
        s_tile[0] = atomicAdd(counter, 1u);
        resolve(s_tile[0], 0);
        s_abort = 0;
        s_peek_tag = 0;
    }
    for (int i = threadIdx.x; i < TILE; i += GCTA) s_cnt[i] = 0xffff0000u;
    __syncthreads();
    // field, first element and element count of local tile tt of a reduction with tpf_ tiles per field
    auto geom = [&](uint32_t tt, uint32_t tpf_, uint32_t E_, uint32_t& f, uint32_t& e0, int& nh) {
        f = tt / tpf_;
        e0 = (tt - f * tpf_) * TILE;
        nh = static_cast<int>(min(static_cast<uint32_t>(TILE), E_ - e0));
    };
    // thread g == 0: element block e of field fi of reduction pi into the stage
    auto issue = [&](const LaunchParams& pi, uint32_t fi, uint32_t e) {
        if (bchk(fi < static_cast<uint32_t>(pi.n_fields) && e < static_cast<uint64_t>(pi.n_elem), &pi.ctl->status))
            bulk_load(stage, pi.fields[fi] + static_cast<uint64_t>(e) * N3, 8u * N3, bar);
    };
    uint32_t parity = 0;
    uint32_t tag = 0;
    bool inflight = false;
    unsigned recomputed = 0;
    uint32_t t_prev = 0xffffffffu;
    int nh_prev = 0, par = 0;
    uint32_t tot_prev = 0;

    // Copy the staged codes of a tile (parity pp, nhp elements, descriptor pd) to code_base + 2
    // (excl + prefix): warp 0 of each group, lane L: the group's element gi + GPC L.
    auto place_codes = [&](const LaunchParams& pd, int pp, int nhp, uint64_t excl) {
        if (wg != 0) return;
        unsigned* status = &pd.ctl->status;
        const uint32_t* pre = stage_pre + pp * (kWarpTile + 1);
        const int16_t* arena = stage_codes + (pp * kWarpCtaWarps + gi * WPE) * kWarpArena;
        const int il = gi + GPC * lane;
        uint32_t b = 0, n = 0, off = kDirect;
        if (il < nhp) {
            b = pre[il];
            n = pre[il + 1] - b;
            off = stage_off[pp * kWarpTile + il];
        }
        const uint64_t gbyte = pd.code_base + 2ull * (excl + b);
        bool copy = off != kDirect && n > 0;
        if (copy && gbyte + 2ull * n > pd.payload_cap) {
            atomicOr(status, static_cast<unsigned>(SEMR_STATUS_OVERFLOW));
            copy = false;
        }
        copy = copy && bchk(off + n <= static_cast<uint32_t>(ARENA) && gbyte >= pd.code_base, status);
        if (copy && n <= 32u) {
            int16_t* dst = reinterpret_cast<int16_t*>(pd.payload + gbyte);
            const int16_t* src = arena + off;
            for (uint32_t k = 0; k < n; ++k) dst[k] = src[k];
        }
        for (uint32_t big = __ballot_sync(FULL, copy && n > 32u); big; big &= big - 1) {
            const int src_lane = __ffs(big) - 1;
            const uint32_t nb = __shfl_sync(FULL, n, src_lane), ob = __shfl_sync(FULL, off, src_lane);
            int16_t* dst = reinterpret_cast<int16_t*>(pd.payload + __shfl_sync(FULL, gbyte, src_lane));
            for (uint32_t k = lane; k < nb; k += 32) dst[k] = arena[ob + k];
        }
    };

    if (s_tile[0] < total_tiles) {  // the first block of each group's first tile
        const LaunchParams* pn = BATCH ? &q.items[s_titem[0]] : &A.p;
        uint32_t f, e0;
        int nh;
        geom(s_tloc[0], static_cast<uint32_t>(pn->tiles_per_field), static_cast<uint32_t>(pn->n_elem), f, e0, nh);
        if (gi < nh) {
            if (g == 0) issue(*pn, f, e0 + gi);
            inflight = true;
        }
    }
    for (;;) {
    // Tiles are claimed only once the previous one is computed, so they start in about the
    // order of their claims and a look-back never waits for a tile not yet begun.
    if (s_tile[0] >= total_tiles) break;
    const uint32_t gtile = s_tile[0];
    const uint32_t item = s_titem[0], tcur = s_tloc[0];  // tcur: the tile's index within its reduction
    if constexpr (BATCH) {  // the item's descriptor into this tile's slot (the other holds the previous one's)
        __syncthreads();    // the slot's last reader (the placement of two tiles ago) is done
        constexpr int PW = sizeof(LaunchParams) / 4;
        static_assert(sizeof(LaunchParams) % 4 == 0, "descriptor copy by words");
        for (int i = threadIdx.x; i < PW; i += GCTA)
            reinterpret_cast<int*>(&s_par[par])[i] = reinterpret_cast<const int*>(&q.items[item])[i];
        __syncthreads();
    }
    const LaunchParams& p = BATCH ? s_par[par] : A.p;
    const LaunchParams& pprev = BATCH ? s_par[par ^ 1] : A.p;
    unsigned* status = &p.ctl->status;
    float tau_h = A.tau_h, tau_l = A.tau_l;
    if constexpr (BATCH) {
        tau_h = static_cast<float>(p.tau);
        tau_l = static_cast<float>(p.tau - static_cast<double>(tau_h));
    }
    const uint32_t E = static_cast<uint32_t>(p.n_elem), tpf = static_cast<uint32_t>(p.tiles_per_field);
    uint32_t f, e0;
    int nh;
    geom(tcur, tpf, E, f, e0, nh);
    int16_t* arena = stage_codes + (par * kWarpCtaWarps + gi * WPE) * kWarpArena;
    uint32_t atop = 0;
    uint8_t* fsec = p.payload + p.header_bytes + static_cast<uint64_t>(f) * p.fixed_bytes;
    const uint64_t mbytes = pad16(static_cast<uint64_t>(E) * MB);
    int16_t* sdst = reinterpret_cast<int16_t*>(fsec + mbytes);
    uint16_t* cdst = reinterpret_cast<uint16_t*>(fsec + mbytes + pad16(2ull * E));
    // bounds build: the field section's layout within the payload (each element also tests e < E)
    const bool fok = bchk(f < static_cast<uint32_t>(p.n_fields) && mbytes + 2 * pad16(2ull * E) <= p.fixed_bytes &&
                              p.header_bytes + (f + 1ull) * p.fixed_bytes <= p.code_base &&
                              p.code_base <= p.payload_cap,
                          status);
    for (int il = gi; il < nh; il += GPC) {
        const uint32_t e = e0 + static_cast<uint32_t>(il);
        const bool eok = fok && bchk(e < E, status);
        bool landed = mbar_wait_bounded(bar, parity);  // uniform over the warp

        // ---- the element's largest high word of |u| (first pass over the stage's high words; if the
        // block did not land the values are meaningless, but every read stays inside the stage)
        // (the pencils' doubles stay in registers for the split below; an absent pencil is 0)
        const double* su = reinterpret_cast<const double*>(stage);
        uint32_t hm = 0;
        uint4 raw[2][LX / 2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int P = s ? P1 : P0;
            const bool ok = s == 0 || v1;
            const uint4* row = reinterpret_cast<const uint4*>(su + P * LX);
#pragma unroll
            for (int c = 0; c < LX / 2; ++c) {
                raw[s][c] = ok ? row[c] : make_uint4(0u, 0u, 0u, 0u);
                hm = max(hm, max(raw[s][c].y & 0x7fffffffu, raw[s][c].w & 0x7fffffffu));
            }
        }
        uint32_t hmax = __reduce_max_sync(FULL, hm);
        if constexpr (WPE > 1) {  // the group's maximum, and whether the block landed for both warps
            if (lane == 0) {
                xu[XH + wg] = hmax;
                xu[XA + wg] = landed ? 1u : 0u;
            }
            gsync<WPE>(gi);
            hmax = max(xu[XH], xu[XH + 1]);
            landed = (xu[XA] & xu[XA + 1]) != 0u;
        }
        if (!landed) {  // a bounded wait gave up (uniform over the group): stop taking work
            if (g == 0) {
                atomicOr(status, static_cast<unsigned>(SEMR_STATUS_TIMEOUT));
                s_abort = 1;
            }
            break;  // inflight stays set: the copy may still land, and the kernel's end waits for it
        }
        parity ^= 1u;
        inflight = false;
        const bool tiny = hmax < 0x00100000u;
        const int ke = tiny ? 0 : min(static_cast<int>(hmax >> 20) - 1023, 1023);
        const int bias = 0x38000000 + (ke << 20);
        if (g == 0) {
            s_res[il].ke = ke;
            s_res[il].hmax = hmax;
        }

        // ---- split both pencils into floats (integer instructions); an absent pencil is 0
        float2 uh[LX], ul[LX];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
#pragma unroll
            for (int c = 0; c < LX / 2; ++c) {
                const uint4 v = raw[s][c];
                const uint32_t lo[2] = {v.x, v.z}, hi[2] = {v.y, v.w};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float vh_, vl_ = 0.0f;
                    if constexpr (DF) w_split(lo[h], hi[h], bias, vh_, vl_);
                    else vh_ = w_d2f_rz(lo[h], hi[h], bias);
                    if (s == 0) {
                        uh[2 * c + h].x = vh_;
                        ul[2 * c + h].x = vl_;
                    } else {
                        uh[2 * c + h].y = vh_;
                        ul[2 * c + h].y = vl_;
                    }
                }
            }
        }

        // FP64 mode at lx = 10 and with cumulative truncation (measured): the thread's energy partial
        // now, and the pencils' low words parked in the group's slots until the errors need them
        // (their registers are free in between)
        constexpr bool PARK = DF && (LX > 6 || CUM);
        constexpr bool PARKH = DF && LX > 6 && !CUM;  // and the high words (after the first contraction)
        f2 sp_e = {0.0f, 0.0f};
        if constexpr (PARK) {
            p2 acc = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
#pragma unroll
            for (int i = 0; i < LX; ++i) {
                const float2 ph = f2mul(uh[i], uh[i]);
                const float2 pl = f2fma(uh[i], f2add(ul[i], ul[i]), f2fma(uh[i], uh[i], f2neg(ph)));
                df_fma_acc2(acc, {A.tab.wh2[i], A.tab.wl2[i]}, {ph, pl});
            }
            acc = df_norm2(acc);
            sp_e = df_add(df_mul({acc.h.x, acc.l.x}, wjk0), df_mul({acc.h.y, acc.l.y}, wjk1));
            float2* sul = reinterpret_cast<float2*>(gsm + SM::o_ul);
#pragma unroll
            for (int i = 0; i < LX; ++i) sul[i * GT + g] = ul[i];
        }

        // ---- forward transform: i in registers, j and k through the group's transposes
        float2 a2[LX];  // coefficient r of the modal pencils (q, p) = P0, P1
        {
            float2 y[LX];
            g_fwd2<LX>(A.tab.A2, uh, y);
            if constexpr (!DF) {  // the FP32 form parks u until the errors
                float2* sul = reinterpret_cast<float2*>(gsm + SM::o_ul);
#pragma unroll
                for (int i = 0; i < LX; ++i) sul[i * GT + g] = uh[i];
            } else if constexpr (PARKH) {  // FP64 mode at lx = 10, threshold truncation: the high words too
                float2* suh = reinterpret_cast<float2*>(gsm + SM::o_uh);
#pragma unroll
                for (int i = 0; i < LX; ++i) suh[i * GT + g] = uh[i];
            }
#pragma unroll
            for (int pp = 0; pp < LX; ++pp) {
                T[k0 * PL + j0 * LP + pp] = y[pp].x;
                if (v1) T[k1 * PL + j1 * LP + pp] = y[pp].y;
            }
            gsync<WPE>(gi);
            // every thread has consumed the stage: request this group's next element
            if (il + GPC < nh) {
                if (g == 0) {
                    fence_proxy_async();
                    issue(p, f, e + GPC);
                }
                inflight = true;
            }
            float2 x[LX];  // pencils (k, p) = (P / LX, P % LX): values over j
#pragma unroll
            for (int jj = 0; jj < LX; ++jj)
                x[jj] = make_float2(T[k0 * PL + jj * LP + j0], v1 ? T[k1 * PL + jj * LP + j1] : 0.0f);
            g_fwd2<LX>(A.tab.A2, x, y);
#pragma unroll
            for (int q = 0; q < LX; ++q) {
                T2[q * PL + k0 * LP + j0] = y[q].x;
                if (v1) T2[q * PL + k1 * LP + j1] = y[q].y;
            }
            gsync<WPE>(gi);
#pragma unroll
            for (int kk = 0; kk < LX; ++kk)  // pencils (q, p) = (P / LX, P % LX): values over k
                x[kk] = make_float2(T2[k0 * PL + kk * LP + j0], v1 ? T2[k1 * PL + kk * LP + j1] : 0.0f);
            g_fwd2<LX>(A.tab.A2, x, a2);
        }

        // ---- element energy S (pencil sums over i with w_i, times w_j w_k) and the mode-ordered layout
        f2 S;
        {
            f2 sp = {0.0f, 0.0f};
            if constexpr (PARK) {
                sp = warp_sum_pair(sp_e);
            } else if constexpr (DF) {
                p2 acc = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
#pragma unroll
                for (int i = 0; i < LX; ++i) {
                    const float2 ph = f2mul(uh[i], uh[i]);
                    const float2 pl = f2fma(uh[i], f2add(ul[i], ul[i]), f2fma(uh[i], uh[i], f2neg(ph)));
                    df_fma_acc2(acc, {A.tab.wh2[i], A.tab.wl2[i]}, {ph, pl});
                }
                acc = df_norm2(acc);
                sp = df_add(df_mul({acc.h.x, acc.l.x}, wjk0), df_mul({acc.h.y, acc.l.y}, wjk1));
                sp = warp_sum_pair(sp);
            } else {
                float2 s2 = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int r = 0; r < LX; ++r) s2 = f2fma(a2[r], a2[r], s2);
                sp.h = warp_sum_f(s2.x + (v1 ? s2.y : 0.0f));
            }
            // the first buffer is free (its last reads were before the second barrier): modes in order
#pragma unroll
            for (int r = 0; r < LX; ++r) {
                M[P0 + NP * r] = a2[r].x;
                if (v1) M[P1 + NP * r] = a2[r].y;
            }
            if constexpr (WPE > 1) {
                if (lane == 0) {
                    xf[XS + wg] = sp.h;
                    xf[XSL + wg] = sp.l;
                }
            }
            gsync<WPE>(gi);
            if constexpr (WPE > 1) {
                sp = df_add({xf[XS], xf[XSL]}, {xf[XS + 1], xf[XSL + 1]});
            }
            S = sp;
        }
        float am[WPW];  // this lane's modes m = 32 (w0 + kk) + lane
        const int w0 = wg * WPW;
#pragma unroll
        for (int kk = 0; kk < WPW; ++kk) {
            const int m = 32 * (w0 + kk) + lane;
            am[kk] = (w0 + kk < MW && m < N3) ? M[m] : 0.0f;
        }

        // ---- t = tau S', step, threshold g (uniform over the group)
        const bool bad = hmax >= (static_cast<uint32_t>(1023 + 500) << 20);
        int emode = 0, step = INT16_MIN, sps = 0;
        f2 t = {0.0f, 0.0f};
        float gth = 0.0f;
        if (bad || !isfinite(S.h)) {
            if (g == 0) atomicOr(status, static_cast<unsigned>(SEMR_STATUS_NONFINITE));
        } else if (tiny) {
            if (g == 0 && hmax != 0u) atomicOr(status, static_cast<unsigned>(SEMR_STATUS_TINY));
        } else {
            t = df_norm(df_mul({tau_h, tau_l}, S));
            const uint32_t tb_ = __float_as_uint(t.h);
            int exs = static_cast<int>(tb_ >> 23) - 126;
            if ((tb_ & 0x7fffffu) == 0u && t.l < 0.0f) --exs;
            const int ex = exs + 2 * ke;
            if (ex > 1024) {
                if (g == 0) atomicOr(status, static_cast<unsigned>(SEMR_STATUS_NONFINITE));
            } else if (ex >= -1021) {
                sps = (exs - 1) >> 1;
                step = sps + ke;
                emode = 1;
                asm("sqrt.approx.f32 %0, %1;" : "=f"(gth) : "f"(t.h));
#pragma unroll 1
                for (int it = 0; it < 4 && !sq_ge(gth, t); ++it) gth = __uint_as_float(__float_as_uint(gth) + 1u);
#pragma unroll 1
                for (int it = 0; it < 4; ++it) {
                    const float pr = __uint_as_float(__float_as_uint(gth) - 1u);
                    if (sq_ge(pr, t)) gth = pr; else break;
                }
            }
        }
        const float qd = pow2f(-sps), qu = pow2f(sps);

        // ---- keep decisions (FP64 mode: exact recomputation of what FP32 cannot settle); only the
        // lane's valid modes (m < lx^3) take part
        uint32_t vm = 0;
#pragma unroll
        for (int kk = 0; kk < WPW; ++kk)
            if (w0 + kk < MW && 32 * (w0 + kk) + lane < N3) vm |= 1u << kk;
        uint32_t kb = 0;
        float Mq = 0.0f;  // FP64 mode: the bound in units of the step (the rounding screen, in the quantisation)
        if constexpr (CUM) {
            if (emode == 1) {
                // cumulative-energy truncation, as the lx = 8 warp kernel: keep every mode above gb
                // (surely a^2 > t), then extract the group's largest remaining |a| one at a time until
                // the sum R of the squares left fits t; FP64 mode takes the result where the FP32 bound
                // settles it, else (and beyond kCumIters extractions) the general path decides
                constexpr int kCumIters = 48;
                float M32 = 0.0f, gb;
                if constexpr (DF) {
                    constexpr float kMarg = (3.0f * (LX / 2 + 2) + 2.0f) * 5.9604645e-8f * 2.8285f * 2.0f;
                    const float umax_e = __uint_as_float(0x3f800000u | ((hmax & 0xfffffu) << 3));
                    M32 = kMarg * umax_e * 1.000002f;
                    gb = gth + (M32 + gth * 2.4e-7f);
                    Mq = M32 * qd * 1.000001f;
                } else {
                    gb = __uint_as_float(__float_as_uint(gth) + 1u);
                }
                uint32_t rem = 0;
                float rs = 0.0f, sa = 0.0f;
#pragma unroll
                for (int kk = 0; kk < WPW; ++kk) {
                    const float x = fabsf(am[kk]);
                    const bool low = ((vm >> kk) & 1u) && x < gb;
                    rem |= (low ? 1u : 0u) << kk;
                    rs = low ? fmaf(x, x, rs) : rs;
                    sa = low ? sa + x : sa;
                }
                float R = warp_sum_f(rs), sabs = warp_sum_f(sa);
                int nrem = static_cast<int>(__reduce_add_sync(FULL, static_cast<unsigned>(__popc(rem))));
                if constexpr (WPE > 1) {
                    if (lane == 0) {
                        xf[XR + wg] = R;
                        xf[XB + wg] = sabs;
                        xu[XN + wg] = static_cast<uint32_t>(nrem);
                    }
                    gsync<WPE>(gi);
                    R = xf[XR] + xf[XR + 1];
                    sabs = xf[XB] + xf[XB + 1];
                    nrem = static_cast<int>(xu[XN] + xu[XN + 1]);
                }
                const float R0 = R;
                int it = 0;
                float v = 0.0f;
                uint32_t gm = 0;
                bool done = R <= t.h, open = false;
                for (;;) {
                    uint32_t mk = 0;
#pragma unroll
                    for (int kk = 0; kk < WPW; ++kk)
                        mk = ((rem >> kk) & 1u) ? max(mk, __float_as_uint(am[kk]) & 0x7fffffffu) : mk;
                    const uint32_t wm = __reduce_max_sync(FULL, mk);
                    bool mine = true;  // this warp holds the one extracted
                    gm = wm;
                    if constexpr (WPE > 1) {
                        if (lane == 0) xu[XM + 2 * (it & 1) + wg] = wm;
                        gsync<WPE>(gi);
                        const uint32_t m0 = xu[XM + 2 * (it & 1)], m1 = xu[XM + 2 * (it & 1) + 1];
                        gm = max(m0, m1);
                        mine = wg == 0 ? m0 == gm : m0 != gm;
                    }
                    if (done) break;
                    if (it == kCumIters || gm == 0u) {
                        open = true;
                        break;
                    }
                    if (mine && lane == __ffs(__ballot_sync(FULL, mk == gm)) - 1) {
                        uint32_t hit = 0;
#pragma unroll
                        for (int kk = 0; kk < WPW; ++kk)
                            hit |= (((rem >> kk) & 1u) && (__float_as_uint(am[kk]) & 0x7fffffffu) == gm ? 1u : 0u) << kk;
                        rem &= ~(hit & (0u - hit));
                    }
                    v = __uint_as_float(gm);
                    R = fmaf(-v, v, R);
                    sabs -= v;
                    --nrem;
                    ++it;
                    done = R <= t.h;
                }
                bool settled = !open;
                if constexpr (DF) {
                    if (settled) {
                        float vk = v;
                        if (it == 0) {  // the smallest kept: the smallest above gb
                            uint32_t mn = 0x7f000000u;
#pragma unroll
                            for (int kk = 0; kk < WPW; ++kk)
                                mn = (((vm & ~rem) >> kk) & 1u) ? min(mn, __float_as_uint(am[kk]) & 0x7fffffffu) : mn;
                            mn = __reduce_min_sync(FULL, mn);
                            if constexpr (WPE > 1) {
                                if (lane == 0) xu[XV + wg] = mn;
                                gsync<WPE>(gi);
                                mn = min(xu[XV], xu[XV + 1]);
                            }
                            vk = __uint_as_float(mn);
                        }
                        const float wn = __uint_as_float(gm);
                        const float rho = R0 * (6e-5f + 1.2e-7f * static_cast<float>(it)) + 2.4e-7f * t.h;
                        const float B = 2.0f * M32 * sabs * 1.0001f + static_cast<float>(nrem) * M32 * M32 + rho;
                        const float d1 = t.h - R;
                        settled = d1 * 0.999999f > B;
                        if (vk < 0x1p126f) {
                            const float lv = fmaxf(vk - M32, 0.0f);
                            settled = settled && (lv * lv * 0.999999f - d1 * 1.000001f) > B &&
                                      (vk - wn) > 2.0f * M32 * 1.000001f + vk * 1.2e-7f;
                        }
                    }
                }
                if (!settled) {
                    kb = g_cum_general<LX, WPE, DF>(M, am, vm, w0, wg, gi, g, P0, P1, v1, xu,
                                                    p.fields[f] + static_cast<uint64_t>(e) * N3, A.tab.A64,
                                                    pow2d(-ke), static_cast<double>(t.h) + static_cast<double>(t.l),
                                                    qd, qu, recomputed);
                } else {
                    const uint32_t vb = __float_as_uint(it ? v : gb);
#pragma unroll
                    for (int kk = 0; kk < WPW; ++kk)
                        kb |= ((__float_as_uint(am[kk]) & 0x7fffffffu) >= vb ? 1u : 0u) << kk;
                    kb &= vm;
                }
            }
        } else if (emode == 1) {
            if constexpr (DF) {
                constexpr float kMarg = (3.0f * (LX / 2 + 2) + 2.0f) * 5.9604645e-8f * 2.8285f * 2.0f;
                const float umax_e = __uint_as_float(0x3f800000u | ((hmax & 0xfffffu) << 3));
                const float Mm = kMarg * umax_e * 1.000002f;
                const float Mg = Mm + gth * 2.4e-7f;
                Mq = Mg * qd;
                uint32_t amb = 0;
#pragma unroll
                for (int kk = 0; kk < WPW; ++kk) {
                    const float aa = fabsf(am[kk]);
                    if (aa >= gth + Mg) kb |= 1u << kk;            // surely kept
                    else if (!(aa < gth - Mg)) amb |= 1u << kk;   // undecided
                }
                kb &= vm;
                amb &= vm;
                if (__any_sync(FULL, amb != 0u)) {
                    kb = g_resolve<LX>(M, w0, amb, kb, p.fields[f] + static_cast<uint64_t>(e) * N3, A.tab.A64,
                                       pow2d(-ke), t, qd, qu, recomputed);
                }
            }  // the FP32 form ballots its threshold test directly below
        }

        // ---- mask words of this warp (ballots), the group's count and this warp's rank base
        uint32_t cw = 0, nzw = 0;
#pragma unroll
        for (int kk = 0; kk < WPW; ++kk) {
            if (w0 + kk < MW) {
                const bool keep = (DF || CUM) ? ((kb >> kk) & 1u) != 0u : (emode == 1 && fabsf(am[kk]) >= gth);
                const uint32_t wv = __ballot_sync(FULL, keep);
                if (lane == 0) bm[w0 + kk] = wv;
                cw += __popc(wv);
                nzw |= (wv != 0u ? 1u : 0u) << kk;
            }
        }
        uint32_t n_e = cw, base = 0;
        if constexpr (WPE > 1) {
            if (lane == 0) xu[XC + wg] = cw;
        }
        gsync<WPE>(gi);  // the bitmap is complete (and the counts exchanged)
        if constexpr (WPE > 1) {
            n_e = xu[XC] + xu[XC + 1];
            base = wg ? xu[XC] : 0u;
        }
        // payload: the element's mask bytes, step and count
        {
            const uint8_t* bmb = reinterpret_cast<const uint8_t*>(bm);
            uint8_t* mdst = fsec + static_cast<uint64_t>(e) * MB;
            for (int b = g; eok && b < MB; b += GT) mdst[b] = bmb[b];
        }
        const bool staged = atop + n_e <= static_cast<uint32_t>(ARENA);
        if (g == 0) {
            if (eok) {
                sdst[e] = static_cast<int16_t>(step);
                cdst[e] = static_cast<uint16_t>(n_e);
            }
            s_cnt[il] = (tag << 16) | n_e;
            stage_off[par * kWarpTile + il] = staged ? atop : kDirect;
        }
        if (e + 1 == E && g < 16 && eok) {  // zero the padding after the mask, step and count sections
            const uint64_t me = static_cast<uint64_t>(E) * MB;
            if (me + g < pad16(me)) fsec[me + g] = 0;
            const uint64_t se = 2ull * E;
            if (se + g < pad16(se)) {
                reinterpret_cast<uint8_t*>(sdst)[se + g] = 0;
                reinterpret_cast<uint8_t*>(cdst)[se + g] = 0;
            }
        }

        // ---- quantise: code = rint(a 2^-s'), ties to even, in mode order
        int16_t* qdst = arena + atop;
        bool qwrite = true;
        if (!staged) {
            // the group's arena is full (extreme inputs only): write at the final place, which needs
            // the tile's exclusive prefix and the counts of the tile's earlier elements
            uint64_t before;
            if (s_peek_tag == gtile + 1u) {
                before = s_peek;
            } else {
                before = lookback_peek(p.tile_state, tcur, status);
                if (g == 0) {
                    s_peek = before;
                    __threadfence_block();
                    s_peek_tag = gtile + 1u;
                }
            }
            uint32_t part = 0;
            for (int jj = lane; jj < il; jj += 32) {
                uint32_t v = 0;
                for (uint32_t it = 0; it < (1u << 22); ++it) {
                    v = *reinterpret_cast<volatile uint32_t*>(&s_cnt[jj]);
                    if ((v >> 16) == tag) break;
                    __nanosleep(64);
                    if (it + 1 == (1u << 22)) atomicOr(status, static_cast<unsigned>(SEMR_STATUS_TIMEOUT));
                }
                part += v & 0xffffu;
            }
            before += __reduce_add_sync(FULL, part);
            const uint64_t gbyte = p.code_base + 2ull * before;
            qwrite = gbyte + 2ull * n_e <= p.payload_cap;
            if (!qwrite && g == 0) atomicOr(status, static_cast<unsigned>(SEMR_STATUS_OVERFLOW));
            qwrite = qwrite && bchk(gbyte >= p.code_base, status);
            qdst = reinterpret_cast<int16_t*>(p.payload + gbyte);
        }
        {
            const uint32_t lt_mask = (1u << lane) - 1u;
            uint32_t run = base;
            while (nzw) {
                const int kk = __ffs(nzw) - 1;
                nzw &= nzw - 1;
                const uint32_t wd = bm[w0 + kk];
                const int m = 32 * (w0 + kk) + lane;  // (within the buffer for every lane)
                float a = M[m];
                if constexpr (DF) {  // a kept mode whose rounding the FP32 bound cannot settle is recomputed
                    const float y = fabsf(a) * qd;
                    const bool ra = ((wd >> lane) & 1u) && fabsf((y - floorf(y)) - 0.5f) <= Mq + y * 1.2e-7f;
                    if (__any_sync(FULL, ra))
                        a = g_settle<LX>(a, ra, M, w0, kk, p.fields[f] + static_cast<uint64_t>(e) * N3, A.tab.A64,
                                         pow2d(-ke), qd, qu, recomputed);
                }
                if ((wd >> lane) & 1u) {
                    const float c = (a * qd + 12582912.0f) - 12582912.0f;  // round half to even (|y| < 2^22)
                    const uint32_t rank = run + __popc(wd & lt_mask);
                    if (qwrite) qdst[rank] = static_cast<int16_t>(c);
                    if (rank < static_cast<uint32_t>(KL)) skl[rank] = make_int2(m, __float_as_int(c));
                }
                run += __popc(wd);
            }
        }
        if (staged) atop += n_e;
        gsync<WPE>(gi);  // the kept list is complete

        // ---- reconstruction u~ of the thread's nodal pencils (pairs in FP64 mode)
        float2 vh[LX], vl[LX];
#pragma unroll
        for (int i = 0; i < LX; ++i) {
            vh[i] = make_float2(0.0f, 0.0f);
            vl[i] = make_float2(0.0f, 0.0f);
        }
        if (n_e <= static_cast<uint32_t>(KL)) {
            // u~(i) = sum over kept modes of B phi_p(x_i), B = c 2^s' phi_q(x_j) phi_r(x_k) per pencil
            if constexpr (DF) {
                // Two passes over the kept list: the modes with p = 0 (phi_0 is constant along the
                // pencil; most kept modes have p = 0) give one pair per pencil that starts every
                // point, and each other mode adds B phi_p(x_i) at the LX points
                auto bcoef = [&](int2 kv) -> p2 {  // B of both pencils as packed pairs
                    const int qq = (kv.x / LX) % LX, rr = kv.x / NP;
                    const float2 cs = f2dup(__int_as_float(kv.y) * qu);  // c 2^s', exact
                    const float2 fjh = make_float2(sPh[j0 * LX + qq], sPh[j1 * LX + qq]);
                    const float2 fjl = make_float2(sPl[j0 * LX + qq], sPl[j1 * LX + qq]);
                    const float2 fkh = make_float2(sPh[k0 * LX + rr], sPh[k1 * LX + rr]);
                    const float2 fkl = make_float2(sPl[k0 * LX + rr], sPl[k1 * LX + rr]);
                    const float2 ph = f2mul(fjh, fkh);
                    const float2 pl = f2add(f2fma(fjh, fkh, f2neg(ph)), f2fma(fjh, fkl, f2mul(fjl, fkh)));
                    const float2 bh = f2mul(ph, cs);
                    return {bh, f2fma(pl, cs, f2fma(ph, cs, f2neg(bh)))};
                };
                p2 c0 = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};  // sum of B over the p = 0 modes
                for (uint32_t tk = 0; tk < n_e; ++tk) {
                    const int2 kv = skl[tk];
                    if (kv.x % LX != 0) continue;
                    const p2 B = bcoef(kv);
                    const p2 sm = two_sum2(c0.h, B.h);
                    c0 = fast_two_sum2(sm.h, f2add(sm.l, f2add(c0.l, B.l)));
                }
                {  // times phi_0, the same at every point
                    p2 v0 = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
                    df_fma_acc2(v0, c0, {f2dup(sPTh[0]), f2dup(sPTl[0])});
#pragma unroll
                    for (int i = 0; i < LX; ++i) {
                        vh[i] = v0.h;
                        vl[i] = v0.l;
                    }
                }
                for (uint32_t tk = 0; tk < n_e; ++tk) {
                    const int2 kv = skl[tk];
                    const int pp = kv.x % LX;
                    if (pp == 0) continue;
                    const p2 B = bcoef(kv);
#pragma unroll
                    for (int i = 0; i < LX; ++i) {
                        p2 acc = {vh[i], vl[i]};
                        df_fma_acc2(acc, B, {f2dup(sPTh[pp * LX + i]), f2dup(sPTl[pp * LX + i])});
                        vh[i] = acc.h;
                        vl[i] = acc.l;
                    }
                }
#pragma unroll
                for (int i = 0; i < LX; ++i) {
                    const p2 nn = df_norm2({vh[i], vl[i]});
                    vh[i] = nn.h;
                    vl[i] = nn.l;
                }
            } else {  // one pass: the FP32 form is faster without the p = 0 split
                for (uint32_t tk = 0; tk < n_e; ++tk) {
                    const int2 kv = skl[tk];
                    const int m = kv.x, pp = m % LX, qq = (m / LX) % LX, rr = m / NP;
                    const float cs = __int_as_float(kv.y) * qu;  // c 2^s', exact
                    const float2 B = make_float2(cs * sPh[j0 * LX + qq] * sPh[k0 * LX + rr],
                                                 cs * sPh[j1 * LX + qq] * sPh[k1 * LX + rr]);
#pragma unroll
                    for (int i = 0; i < LX; ++i) vh[i] = f2fma(B, f2dup(sPTh[pp * LX + i]), vh[i]);
                }
            }
        } else {
            // dense inverse (many kept modes): the kept values (code 2^s', else 0) in mode order, then
            // r -> k, q -> j, p -> i through the group's buffer (one float2 buffer, barriers between)
#pragma unroll
            for (int kk = 0; kk < WPW; ++kk) {
                const int m = 32 * (w0 + kk) + lane;
                if (w0 + kk < MW && m < N3) {
                    const bool k = (bm[w0 + kk] >> lane) & 1u;
                    M[m] = k ? ((M[m] * qd + 12582912.0f) - 12582912.0f) * qu : 0.0f;
                }
            }
            gsync<WPE>(gi);
            float2* Tb = reinterpret_cast<float2*>(T);  // [plane][row][col] pairs (h, l) of one pencil value
            if constexpr (DF) {
                p2 x[LX], y[LX];
#pragma unroll
                for (int r = 0; r < LX; ++r)
                    x[r] = {make_float2(M[P0 + NP * r], v1 ? M[P1 + NP * r] : 0.0f), make_float2(0.0f, 0.0f)};
                gsync<WPE>(gi);
                g_inv_df2<LX>(A.tab.Ph, A.tab.Pl, x, y);  // pencil (q, p): values over k
#pragma unroll
                for (int kk = 0; kk < LX; ++kk) {
                    Tb[kk * PL + k0 * LP + j0] = make_float2(y[kk].h.x, y[kk].l.x);
                    if (v1) Tb[kk * PL + k1 * LP + j1] = make_float2(y[kk].h.y, y[kk].l.y);
                }
                gsync<WPE>(gi);
#pragma unroll
                for (int q = 0; q < LX; ++q) {  // pencil (k, p) = (P / LX, P % LX): values over q
                    const float2 a0 = Tb[k0 * PL + q * LP + j0];
                    const float2 a1 = v1 ? Tb[k1 * PL + q * LP + j1] : make_float2(0.0f, 0.0f);
                    x[q] = {make_float2(a0.x, a1.x), make_float2(a0.y, a1.y)};
                }
                gsync<WPE>(gi);
                g_inv_df2<LX>(A.tab.Ph, A.tab.Pl, x, y);  // values over j
#pragma unroll
                for (int jj = 0; jj < LX; ++jj) {
                    Tb[k0 * PL + jj * LP + j0] = make_float2(y[jj].h.x, y[jj].l.x);
                    if (v1) Tb[k1 * PL + jj * LP + j1] = make_float2(y[jj].h.y, y[jj].l.y);
                }
                gsync<WPE>(gi);
#pragma unroll
                for (int pp = 0; pp < LX; ++pp) {  // pencil (k, j) = (P / LX, P % LX): values over p
                    const float2 a0 = Tb[k0 * PL + j0 * LP + pp];
                    const float2 a1 = v1 ? Tb[k1 * PL + j1 * LP + pp] : make_float2(0.0f, 0.0f);
                    x[pp] = {make_float2(a0.x, a1.x), make_float2(a0.y, a1.y)};
                }
                g_inv_df2<LX>(A.tab.Ph, A.tab.Pl, x, y);
#pragma unroll
                for (int i = 0; i < LX; ++i) {
                    vh[i] = y[i].h;
                    vl[i] = y[i].l;
                }
            } else {
                float2 x[LX], y[LX];
#pragma unroll
                for (int r = 0; r < LX; ++r) x[r] = make_float2(M[P0 + NP * r], v1 ? M[P1 + NP * r] : 0.0f);
                gsync<WPE>(gi);
                g_inv2<LX>(A.tab.Ph, x, y);
#pragma unroll
                for (int kk = 0; kk < LX; ++kk) {
                    Tb[kk * PL + k0 * LP + j0] = make_float2(y[kk].x, 0.0f);
                    if (v1) Tb[kk * PL + k1 * LP + j1] = make_float2(y[kk].y, 0.0f);
                }
                gsync<WPE>(gi);
#pragma unroll
                for (int q = 0; q < LX; ++q)
                    x[q] = make_float2(Tb[k0 * PL + q * LP + j0].x, v1 ? Tb[k1 * PL + q * LP + j1].x : 0.0f);
                gsync<WPE>(gi);
                g_inv2<LX>(A.tab.Ph, x, y);
#pragma unroll
                for (int jj = 0; jj < LX; ++jj) {
                    Tb[k0 * PL + jj * LP + j0] = make_float2(y[jj].x, 0.0f);
                    if (v1) Tb[k1 * PL + jj * LP + j1] = make_float2(y[jj].y, 0.0f);
                }
                gsync<WPE>(gi);
#pragma unroll
                for (int pp = 0; pp < LX; ++pp)
                    x[pp] = make_float2(Tb[k0 * PL + j0 * LP + pp].x, v1 ? Tb[k1 * PL + j1 * LP + pp].x : 0.0f);
                g_inv2<LX>(A.tab.Ph, x, y);
#pragma unroll
                for (int i = 0; i < LX; ++i) vh[i] = y[i];
            }
        }

        // ---- errors of the thread's points: e2 = sum w (u - u~)^2, Linf = max |u - u~|
        f2 e2;
        float lh = 0.0f, ll = 0.0f;
        if constexpr (DF) {
            if constexpr (PARK) {
                const float2* sul = reinterpret_cast<const float2*>(gsm + SM::o_ul);
#pragma unroll
                for (int ii = 0; ii < LX; ++ii) ul[ii] = sul[ii * GT + g];
            }
            if constexpr (PARKH) {
                const float2* suh = reinterpret_cast<const float2*>(gsm + SM::o_uh);
#pragma unroll
                for (int ii = 0; ii < LX; ++ii) uh[ii] = suh[ii * GT + g];
            }
            p2 acc = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
            float dm = 0.0f;
#pragma unroll
            for (int i = 0; i < LX; ++i) {
                const p2 d = df_sub2({uh[i], ul[i]}, {vh[i], vl[i]});
                const float2 ph = f2mul(d.h, d.h);
                const float2 pl = f2fma(d.h, f2add(d.l, d.l), f2fma(d.h, d.h, f2neg(ph)));
                df_fma_acc2(acc, {A.tab.wh2[i], A.tab.wl2[i]}, {ph, pl});
                dm = fmaxf(dm, fmaxf(fabsf(d.h.x), v1 ? fabsf(d.h.y) : 0.0f));
            }
            acc = df_norm2(acc);
            e2 = warp_sum_pair(df_add(df_mul({acc.h.x, acc.l.x}, wjk0), df_mul({acc.h.y, acc.l.y}, wjk1)));
            // Linf = max |d| over normalised pairs, ordered by (|dh|, low word signed like dh): within the
            // warp the largest |dh|, then the largest signed low word among the points that attain it
            const float LH = warp_max_nonneg(dm);
            float lbest = -FLT_MAX;
            if (dm == LH) {
#pragma unroll
                for (int i = 0; i < LX; ++i) {
                    const p2 d = df_sub2({uh[i], ul[i]}, {vh[i], vl[i]});
                    if (fabsf(d.h.x) == LH)
                        lbest = fmaxf(lbest, __uint_as_float(__float_as_uint(d.l.x) ^ (__float_as_uint(d.h.x) & 0x80000000u)));
                    if (v1 && fabsf(d.h.y) == LH)
                        lbest = fmaxf(lbest, __uint_as_float(__float_as_uint(d.l.y) ^ (__float_as_uint(d.h.y) & 0x80000000u)));
                }
            }
            const uint32_t key = (dm == LH) ? (__float_as_uint(lbest) ^ ((__float_as_uint(lbest) >> 31) ? 0xffffffffu : 0x80000000u)) : 0u;
            const uint32_t kmax = __reduce_max_sync(FULL, key);
            lh = LH;
            ll = (LH == 0.0f) ? 0.0f : __uint_as_float((kmax >> 31) ? (kmax ^ 0x80000000u) : ~kmax);
        } else {
            {
                const float2* sul = reinterpret_cast<const float2*>(gsm + SM::o_ul);
#pragma unroll
                for (int ii = 0; ii < LX; ++ii) uh[ii] = sul[ii * GT + g];
            }
            float2 acc = make_float2(0.0f, 0.0f);
            float dm = 0.0f;
#pragma unroll
            for (int i = 0; i < LX; ++i) {
                const float2 d = f2sub(uh[i], vh[i]);
                acc = f2fma(f2mul(A.tab.wh2[i], d), d, acc);
                dm = fmaxf(dm, fmaxf(fabsf(d.x), v1 ? fabsf(d.y) : 0.0f));
            }
            e2 = {warp_sum_f(fmaf(acc.x, wjk0.h, v1 ? acc.y * wjk1.h : 0.0f)), 0.0f};
            lh = warp_max_nonneg(dm);
        }
        if constexpr (WPE > 1) {  // the group's sums and maxima
            if (lane == 0) {
                xf[XE + wg] = e2.h;
                xf[XEL + wg] = e2.l;
                xf[XL + wg] = lh;
                xf[XLL + wg] = ll;
            }
            gsync<WPE>(gi);
            e2 = df_add({xf[XE], xf[XEL]}, {xf[XE + 1], xf[XEL + 1]});
            const float h0 = xf[XL], h1 = xf[XL + 1], l0 = xf[XLL], l1 = xf[XLL + 1];
            lh = fmaxf(h0, h1);
            ll = (h0 > h1) ? l0 : (h1 > h0) ? l1 : fmaxf(l0, l1);
        }
        if (p.write_recon && p.recon[f] && eok) {  // u~ = u~' 2^ke (exact)
            const double sc = pow2d(ke);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                if (s == 1 && !v1) continue;
                double* dst = p.recon[f] + static_cast<uint64_t>(e) * N3 + (s ? P1 : P0) * LX;
#pragma unroll
                for (int i = 0; i < LX; ++i) {
                    const float h = s ? vh[i].y : vh[i].x, l = s ? vl[i].y : vl[i].x;
                    dst[i] = (static_cast<double>(h) + static_cast<double>(l)) * sc;
                }
            }
        }
        if (g == 0) {
            GStash& st = s_res[il];
            st.sh = tiny ? 0.0f : S.h;
            st.sl = tiny ? 0.0f : S.l;
            st.eh = tiny ? 0.0f : e2.h;
            st.el = tiny ? 0.0f : e2.l;
            st.lh = tiny ? 0.0f : lh;
            st.ll = tiny ? 0.0f : ll;
        }
        gsync<WPE>(gi);  // the group's buffers and exchange slots are reused by the next element
    }
    if (threadIdx.x == 0) {
        s_tile[1] = atomicAdd(counter, 1u);
        resolve(s_tile[1], 1);
    }
    __syncthreads();  // every element of the tile is done
    if (s_tile[1] < total_tiles && !s_abort) {  // each group's first block of the next tile
        const LaunchParams* pn = BATCH ? &q.items[s_titem[1]] : &A.p;
        uint32_t fn, e0n;
        int nhn;
        geom(s_tloc[1], static_cast<uint32_t>(pn->tiles_per_field), static_cast<uint32_t>(pn->n_elem), fn, e0n, nhn);
        if (gi < nhn) {
            if (g == 0) {
                fence_proxy_async();
                issue(*pn, fn, e0n + gi);
            }
            inflight = true;
        }
    }
    constexpr int EPL = (TILE + 31) / 32;  // tile bookkeeping: elements per lane of warp 0
    if (wid == 0) {
        uint32_t cl[EPL], c = 0;
#pragma unroll
        for (int h = 0; h < EPL; ++h) {
            const int ii = EPL * lane + h;
            cl[h] = (ii < nh) ? (s_cnt[ii] & 0xffffu) : 0u;
            c += cl[h];
        }
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        uint32_t* pre = stage_pre + par * (kWarpTile + 1);
        uint32_t run = incl - c;
#pragma unroll
        for (int h = 0; h < EPL; ++h) {
            if (EPL * lane + h < TILE) pre[EPL * lane + h] = run;
            run += cl[h];
        }
        const uint32_t tot = __shfl_sync(FULL, incl, 31);
        if (lane == 0 && bchk(tcur < static_cast<uint32_t>(p.n_fields) * tpf && nh <= kWarpTile, status)) {
            pre[nh] = tot;
            st_release_u64(&p.tile_state[tcur], (tcur == 0 ? kFlagPrefix : kFlagAggregate) | tot);
        }
        if (t_prev != 0xffffffffu) {
            const uint64_t excl = lookback_warp(pprev.tile_state, t_prev, tot_prev, &pprev.ctl->status);
            if (lane == 0) s_excl = excl;
        }
        tot_prev = tot;
    } else if (wid == 2 && lane == 0) {
        s_tile[0] = s_tile[1];
        s_titem[0] = s_titem[1];
        s_tloc[0] = s_tloc[1];
    }
    {  // every warp: FP64 partials and element report of the elements wid + 4 lane
        double v0 = 0.0, v1d = 0.0;
        unsigned long long m2 = 0ull, m3 = 0ull;
        const int il = wid + 4 * lane;
        if (il < nh) {
            const GStash st = s_res[il];
            const uint64_t ge = static_cast<uint64_t>(f) * E + e0 + il;
            const double J = p.jac[e0 + il];
            const double sc = pow2d(st.ke);
            const double Sd = ((static_cast<double>(st.sh) + static_cast<double>(st.sl)) * sc) * sc;
            const double e2d = ((static_cast<double>(st.eh) + static_cast<double>(st.el)) * sc) * sc;
            v0 = J * e2d;
            v1d = J * Sd;
            const double x2 = (static_cast<double>(st.lh) + static_cast<double>(st.ll)) * sc;
            m2 = static_cast<unsigned long long>(__double_as_longlong(x2));
            m3 = st.hmax;
            const bool gok = bchk(ge < static_cast<uint64_t>(p.n_fields) * E, status);
            if (gok) p.hmax_elem[ge] = st.hmax;
            if (p.elem_report && gok) {
                double* er = p.elem_report + 3 * ge;
                er[0] = v0;
                er[1] = v1d;
                er[2] = x2;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v0 += __shfl_down_sync(FULL, v0, o);
            v1d += __shfl_down_sync(FULL, v1d, o);
            m2 = max(m2, __shfl_down_sync(FULL, m2, o));
            m3 = max(m3, __shfl_down_sync(FULL, m3, o));
        }
        if (lane == 0) {
            s_wpart[wid][0] = v0;
            s_wpart[wid][1] = v1d;
            s_wpart[wid][2] = __longlong_as_double(static_cast<long long>(m2));
            s_wpart[wid][3] = static_cast<double>(m3);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && bchk(tcur < static_cast<uint32_t>(p.n_fields) * tpf, status)) {
        double* tp = p.tile_part + 4ull * tcur;
        tp[0] = ((s_wpart[0][0] + s_wpart[1][0]) + s_wpart[2][0]) + s_wpart[3][0];
        tp[1] = ((s_wpart[0][1] + s_wpart[1][1]) + s_wpart[2][1]) + s_wpart[3][1];
        tp[2] = fmax(fmax(s_wpart[0][2], s_wpart[1][2]), fmax(s_wpart[2][2], s_wpart[3][2]));
        tp[3] = fmax(fmax(s_wpart[0][3], s_wpart[1][3]), fmax(s_wpart[2][3], s_wpart[3][3]));
    }
    if (t_prev != 0xffffffffu) place_codes(pprev, par ^ 1, nh_prev, s_excl);
    if (recomputed && lane == 0) atomicAdd(&p.ctl->recomputed, recomputed);
    recomputed = 0;
    t_prev = tcur;
    nh_prev = nh;
    par ^= 1;
    if (s_abort) break;
    tag = (tag + 1 == 0xffffu) ? 0u : tag + 1;
    __syncthreads();
    }
    if (t_prev != 0xffffffffu && !s_abort) {  // the last tile: its look-back, then its codes
        const LaunchParams& pl = BATCH ? s_par[par ^ 1] : A.p;
        if (wid == 0) {
            const uint64_t excl = lookback_warp(pl.tile_state, t_prev, tot_prev, &pl.ctl->status);
            if (lane == 0) s_excl = excl;
        }
        __syncthreads();
        place_codes(pl, par ^ 1, nh_prev, s_excl);
    }
    // after an abort: let a requested block land before the CTA exits (the second, bounded wait)
    if (inflight) drain_stage(bar, parity, &(BATCH ? s_par[par ^ 1] : A.p).ctl->status);
    // a single launch finalizes in the CTA that finishes last (no separate kernel, which could wait
    // behind another launch's persistent CTAs), one field per warp
    if constexpr (!BATCH) {
        if (last_cta_done(&A.p.ctl->done_ctas))
            for (int f = wid; f < A.p.n_fields; f += GCTA / 32) finalize_field_warp(A.p, f, LX, TILE);
    }
}

// One warp per (item, field) of a batched launch, eight per block: the fixed-order finalize of a
// single launch's last CTA, so a batched snapshot's reports equal its single launch's bit for bit.
template <int LX>
__global__ void __launch_bounds__(256) finalize_group_batch_kernel(const BatchQueue q, uint32_t total_fields) {
    const uint32_t gf = blockIdx.x * 8u + (threadIdx.x >> 5);
    if (gf >= total_fields) return;  // uniform over the warp
    int lo = 0, hi = q.n_items - 1;  // last item with field_base <= gf
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (q.field_base[mid] <= gf) lo = mid; else hi = mid - 1;
    }
    finalize_field_warp(q.items[lo], static_cast<int>(gf - q.field_base[lo]), LX, GCfg<LX>::TILE);
}

template <int LX>
GTables<LX> make_gtables() {
    GTables<LX> t;
    double Am[LX * LX], Phi[LX * LX], w[LX];
    basis_tables(LX, Am, Phi, w);
    for (int i = 0; i < LX * LX; ++i) {
        const float ah = static_cast<float>(Am[i]);
        t.A2[i] = make_float2(ah, ah);
        t.A64[i] = Am[i];
        t.Ph[i] = static_cast<float>(Phi[i]);
        t.Pl[i] = static_cast<float>(Phi[i] - static_cast<double>(t.Ph[i]));
    }
    for (int i = 0; i < LX; ++i) {
        t.wh[i] = static_cast<float>(w[i]);
        t.wl[i] = static_cast<float>(w[i] - static_cast<double>(t.wh[i]));
        t.wh2[i] = make_float2(t.wh[i], t.wh[i]);
        t.wl2[i] = make_float2(t.wl[i], t.wl[i]);
    }
    return t;
}

// Launch of one reduction (q empty) or of a batch queue (BATCH; p unused but for stage_ctas).
template <int LX, int MODE, bool BATCH, bool CUM = false>
int launch_group_mode(const LaunchParams& p, const BatchQueue& q, uint64_t stage_ctas, void* stream) {
    using SM = GSmem<LX, MODE != 0, CUM>;
    GArgs<LX> a;
    std::memset(&a, 0, sizeof(a));
    a.tab = make_gtables<LX>();
    if (!BATCH) {
        a.p = p;
        a.tau_h = static_cast<float>(p.tau);
        a.tau_l = static_cast<float>(p.tau - static_cast<double>(a.tau_h));
        a.total_tiles = static_cast<uint32_t>(static_cast<uint64_t>(p.n_fields) * p.tiles_per_field);
    }
    const uint64_t total = BATCH ? q.total_tiles : a.total_tiles;
    cudaError_t err;
    auto kern = reduce_group_kernel<LX, MODE, BATCH, CUM>;
    if ((err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes)) != cudaSuccess)
        return (int)err;
    int dev = 0, sms = 0, per_sm = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return (int)err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GCTA, SM::bytes)) != cudaSuccess)
        return (int)err;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    // persistent: as many CTAs as fit at once, never more than tiles or staging slots
    const uint64_t want = std::min<uint64_t>(total, stage_ctas);
    const unsigned grid = (unsigned)std::min<uint64_t>(want, static_cast<uint64_t>(sms) * per_sm);
    if (grid == 0) return (int)cudaErrorInvalidConfiguration;
    kern<<<grid, GCTA, SM::bytes, static_cast<cudaStream_t>(stream)>>>(a, q);
    return (int)cudaGetLastError();
}

}  // namespace

int group_tile(int lx) {
    switch (lx) {
        case 6: return GCfg<6>::TILE;
        case 10: return GCfg<10>::TILE;
        default: return 0;
    }
}

bool group_applicable(const LaunchParams& p) {
    if (group_tile(p.lx) == 0 || p.lossless || p.width != 2) return false;
    if (p.precision != SEMR_FP64 && p.precision != SEMR_FP32) return false;
    for (int f = 0; f < p.n_fields; ++f)
        if (reinterpret_cast<uintptr_t>(p.fields[f]) & 15u) return false;  // bulk copies need 16-byte aligned blocks
    return true;
}

int launch_reduce_group(const LaunchParams& p, void* stream) {
    const bool df = p.precision != SEMR_FP32;
    const BatchQueue q{};
    const uint64_t sc = static_cast<uint64_t>(p.stage_ctas);
    if (p.cumulative) {  // cumulative-energy truncation (single launches only)
        switch (p.lx) {
            case 6: return df ? launch_group_mode<6, 1, false, true>(p, q, sc, stream)
                              : launch_group_mode<6, 0, false, true>(p, q, sc, stream);
            case 10: return df ? launch_group_mode<10, 1, false, true>(p, q, sc, stream)
                               : launch_group_mode<10, 0, false, true>(p, q, sc, stream);
            default: return (int)cudaErrorInvalidValue;
        }
    }
    switch (p.lx) {
        case 6: return df ? launch_group_mode<6, 1, false>(p, q, sc, stream) : launch_group_mode<6, 0, false>(p, q, sc, stream);
        case 10: return df ? launch_group_mode<10, 1, false>(p, q, sc, stream) : launch_group_mode<10, 0, false>(p, q, sc, stream);
        default: return (int)cudaErrorInvalidValue;
    }
}

int launch_reduce_group_batch(const BatchQueue& q, int lx, int precision, bool cumulative, uint64_t stage_ctas,
                              void* stream) {
    const bool df = precision != SEMR_FP32;
    LaunchParams p;
    std::memset(&p, 0, sizeof(p));
    if (cumulative) {
        switch (lx) {
            case 6: return df ? launch_group_mode<6, 1, true, true>(p, q, stage_ctas, stream)
                              : launch_group_mode<6, 0, true, true>(p, q, stage_ctas, stream);
            case 10: return df ? launch_group_mode<10, 1, true, true>(p, q, stage_ctas, stream)
                               : launch_group_mode<10, 0, true, true>(p, q, stage_ctas, stream);
            default: return (int)cudaErrorInvalidValue;
        }
    }
    switch (lx) {
        case 6: return df ? launch_group_mode<6, 1, true>(p, q, stage_ctas, stream) : launch_group_mode<6, 0, true>(p, q, stage_ctas, stream);
        case 10: return df ? launch_group_mode<10, 1, true>(p, q, stage_ctas, stream) : launch_group_mode<10, 0, true>(p, q, stage_ctas, stream);
        default: return (int)cudaErrorInvalidValue;
    }
}

int launch_finalize_group_batch(const BatchQueue& q, int lx, uint32_t total_fields, void* stream) {
    switch (lx) {
        case 6: finalize_group_batch_kernel<6><<<(total_fields + 7) / 8, 256, 0, static_cast<cudaStream_t>(stream)>>>(q, total_fields); break;
        case 10: finalize_group_batch_kernel<10><<<(total_fields + 7) / 8, 256, 0, static_cast<cudaStream_t>(stream)>>>(q, total_fields); break;
        default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}


}  // namespace semr
