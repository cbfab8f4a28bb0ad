// Warp-per-element fused reduce kernel for lx = 8 (arXiv 2407.20731, Sec. IV-B:
// JPEG-like truncation of the modal Legendre coefficients of SEM element
// blocks, keeping the most energetic modes; Eq. 1 for the compression ratio).
//
// One warp reduces one element-field (an 8^3 block, 4 KB of FP64) at a time.
// A CTA of four warps claims look-back tiles of 128 consecutive elements of one
// field from a global counter (warp w takes elements w, w + 4, ...), and no CTA
// barrier runs per element:
//   * TMA: the block arrives in the warp's shared-memory stage as a 2-D tile
//     (64 pencils x 8 doubles, 64-byte swizzle), so every lane reads its two
//     pencils with conflict-free 16-byte loads; the warp's next block is
//     requested as soon as these values are in registers and streams in meanwhile;
//   * lane L owns the pencils P = L and L + 32 (P = j + 8k) in every phase, the
//     two packed as FP32x2: the forward transform contracts i in registers, then
//     j and k after two padded transposes in shared memory private to the warp;
//     the inverse runs the other way round, so each lane ends with the pencils
//     it loaded;
//   * coefficient a[r][q][p] of mode m = p + 8q + 64r lands in lane m & 31,
//     slot (m >> 5) & 1, register r: each of the 16 ballots over (slot, r) is
//     exactly mask word m >> 5 of the payload;
//   * element sums are warp shuffles; each warp stages its codes in its own
//     arena; at the end of a tile the CTA publishes the tile's code count, then
//     resolves the previous tile's prefix (decoupled look-back, one tile late,
//     so it rarely waits) and copies that tile's staged codes to their place;
//   * the elements' norm partials are kept per tile and converted to FP64 by all
//     lanes at once: B300's FP64 pipe runs at ~1/64 of the FP32 rate, so no FP64
//     instruction runs per point or per element.
//   * the CTA that finishes last (a counter in the scratch control block)
//     computes the field reports, one field per warp, so a single reduction is
//     one launch; a batched launch leaves them to a finalize kernel.
// Precision modes as in semr_fast.cu: SEMR_FP32 runs FP32 transforms with an
// exact float-pair threshold test; SEMR_FP64 runs the forward transform in
// FP32 under a proven error bound, recomputes in hardware FP64 every
// coefficient whose keep or rounding decision that bound cannot settle, and
// does the energy, reconstruction and error norms in float pairs.  Every
// element is read as u 2^-ke (an exact power-of-two prescale, ke the binary
// exponent of its largest |u|).  CUM selects the cumulative-energy truncation:
// the modes above sqrt(t) are kept and the largest remaining |a| extracted one
// at a time until the squares left fit the budget t; FP64 mode keeps that
// answer where the FP32 bound settles it and otherwise takes a general path
// (the element in hardware FP64, a bisection on 64-bit fixed-point energies).
#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched at run time)
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "semr_device.cuh"
#include "semr_warp_common.cuh"

namespace semr {
namespace {

constexpr int WLX = 8, WNP = 64, WN3 = 512;
constexpr int WPB = kWarpCtaWarps;   // warps per CTA
constexpr int TSK = 104, TSJ = 12;   // FP32 transpose strides (plane, row) in floats
constexpr int TSK2 = 72, TSJ2 = 9;   // float-pair transpose strides (dense inverse, FP64 mode)
// sparse reconstruction up to this many kept modes (the capacity of the kept list)
template <bool DF> __host__ __device__ constexpr int wsparse() { return DF ? 24 : 16; }

struct WTables {         // lx = 8 tables, as kernel parameters (constant bank)
    float2 A2[64];         // analysis A[p][i] (hi), duplicated for the packed transforms
    float Ah[64], Al[64];  // analysis A[p][i] (hi, lo)
    float Ph[64], Pl[64];  // synthesis Phi[i][p] (hi, lo)
    float wh[8], wl[8];    // GLL weights (hi, lo)
    float2 w2[8];          // GLL weights (hi), duplicated for the packed FP32 error sums
    double A64[64];        // analysis A[p][i] in FP64 (the exact recomputation)
};

struct WStash {    // one element's results, kept until the end of its tile
    int32_t ke;     // the element's prescale exponent: the values below are those of u 2^-ke
    uint32_t hmax;  // largest high word of |u| (orders the elements like max |u|)
    float sh, sl;   // S = sum w u^2 (pair; FP32 form: sl = 0)
    float eh, el;   // e2 = sum w (u - u~)^2 (pair)
    float lh, ll;   // Linf = max |u - u~| (pair)
};
static_assert(sizeof(WStash) == 32, "stash entry");

struct WArgs {
    CUtensorMap tm[SEMR_MAX_FIELDS];  // one 2-D map per field: [n_elem * 64 pencils][8 doubles]
    LaunchParams p;
    WTables tab;
    float tau_h, tau_l;  // tau as a float pair
    uint32_t n_elem;
    uint32_t tiles_per_field;  // ceil(n_elem / kWarpTile)
    uint32_t total_tiles;      // n_fields * tiles_per_field
};

template <bool DF>
struct WSmem {
    static constexpr size_t stage = 4096;                 // one element block per warp
    static constexpr size_t off_tab = WPB * stage;        // Phi^T (hi, lo), A (hi, lo): 4 x 64 floats
    static constexpr size_t off_dup = off_tab + 1024;     // Phi^T duplicated (hi[, lo]): 64 float2 each
    static constexpr size_t off_wq = off_dup + (DF ? 1024 : 512);  // weight products
    // per-element results of the tile; the FP32 form reads its weight products into registers
    // once, so there they overlay the table
    static constexpr size_t off_res = DF ? off_wq + 8 * 512 : off_wq;
    static constexpr size_t off_warp = off_res + (DF ? sizeof(WStash) * kWarpTile
                                                     : (sizeof(WStash) * kWarpTile > 4 * 512 ? sizeof(WStash) * kWarpTile : 4 * 512));
    // per warp
    static constexpr size_t o_tb = 0;
    static constexpr size_t tb_bytes = DF ? 8 * 8 * TSK2 : 4 * 8 * TSK;
    static constexpr size_t o_mask = o_tb + tb_bytes;     // 16 mask words
    static constexpr size_t o_kl = o_mask + 64;           // kept list (mode, code)
    static constexpr size_t o_bar = o_kl + 8 * wsparse<DF>();
    static constexpr size_t o_ul = (o_bar + 16 + 15) / 16 * 16;  // FP64 mode: parked low words [8][32] float2
    static constexpr size_t wbytes = DF ? o_ul + 8 * 8 * 32 : o_bar + 16;
    static constexpr size_t bytes = off_warp + WPB * wbytes + 512;  // + alignment slack
};
static_assert(8 * 8 * TSK2 >= 4 * 8 * TSK, "pair buffer holds the FP32 one");

// Request `bytes` into dst from the 2-D tensor map at (x, y); completion on bar.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar,
                                            uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// 8-point even-odd folded forward transform of both pencils (coefficients duplicated (A, A)).
__device__ __forceinline__ void w_fwd2(const float2* __restrict__ A2, const float2 (&x)[8], float2 (&y)[8]) {
    const float2 e0 = f2add(x[0], x[7]), e1 = f2add(x[1], x[6]), e2 = f2add(x[2], x[5]), e3 = f2add(x[3], x[4]);
    const float2 o0 = f2sub(x[0], x[7]), o1 = f2sub(x[1], x[6]), o2 = f2sub(x[2], x[5]), o3 = f2sub(x[3], x[4]);
#pragma unroll
    for (int p = 0; p < 8; p += 2) {
        y[p] = f2fma(A2[p * 8 + 3], e3, f2fma(A2[p * 8 + 2], e2, f2fma(A2[p * 8 + 1], e1, f2mul(A2[p * 8], e0))));
        y[p + 1] = f2fma(A2[p * 8 + 11], o3,
                         f2fma(A2[p * 8 + 10], o2, f2fma(A2[p * 8 + 9], o1, f2mul(A2[p * 8 + 8], o0))));
    }
}

// Coefficient (s, r) = (w & 1, w >> 1) of a lane, for a warp-uniform mask word w.
__device__ __forceinline__ float pick(const float2 (&a)[8], int w) {
    switch (w) {
        case 0: return a[0].x;
        case 1: return a[0].y;
        case 2: return a[1].x;
        case 3: return a[1].y;
        case 4: return a[2].x;
        case 5: return a[2].y;
        case 6: return a[3].x;
        case 7: return a[3].y;
        case 8: return a[4].x;
        case 9: return a[4].y;
        case 10: return a[5].x;
        case 11: return a[5].y;
        case 12: return a[6].x;
        case 13: return a[6].y;
        case 14: return a[7].x;
        default: return a[7].y;
    }
}

// Exact coefficient a'[r][q][p] = 2^-ke sum A[r][k] A[q][j] A[p][i] u[k][j][i] of the element block
// at `u` (global memory, [pencil][8]) in hardware FP64: each lane contracts its two pencils
// (k0 + 4s, j) with A[p][.], A[q][j], A[r][k] and the warp sums them.  FP64 because the decisions
// sent here can lie within 1e-8 of a tie in relative terms: a kept coefficient may be as small as
// about 7e-6 max|u| at tau = 1e-6 in a spiky element, where float pairs (47 input bits) would
// carry a relative error near 1e-8.  Rare (decisions the FP32 bound cannot settle), so the slow
// FP64 pipe costs little: out of line, and the block is reread from global memory (it was just
// loaded, so L2 holds it) rather than from the stage, which already receives the warp's next block.
__device__ __noinline__ double exact_coef(const double* __restrict__ u, int pp, int qq, int rr,
                                          const double* __restrict__ A64, double sc) {
    const int lane = threadIdx.x & 31, j = lane & 7, k0 = lane >> 3;
    double c = 0.0;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const double2* row = reinterpret_cast<const double2*>(u + (lane + 32 * s) * 8);
        double xs = 0.0;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            const double2 v = __ldg(row + cc);
            xs = fma(A64[pp * 8 + 2 * cc], v.x, xs);
            xs = fma(A64[pp * 8 + 2 * cc + 1], v.y, xs);
        }
        c = fma(xs * A64[qq * 8 + j], A64[rr * 8 + k0 + 4 * s], c);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    return c * sc;
}

// Settles every ambiguous keep or rounding decision of an element exactly (a rare path,
// out of line): the lane's coefficients (s, r) are at buf[lane * 17 + 8 s + r]; each mode
// with its bit set in the lane's amb is recomputed exactly, one at a time over the warp, and
// a kept one becomes its code times 2^s (exact), so the quantisation reproduces the code of
// the exact value.  Returns the lane's updated keep bits.  keep_fixed: the keep bits are
// already exact (cumulative truncation) and only the roundings are settled.
__device__ __noinline__ uint32_t resolve_ambiguous(float* buf, uint32_t amb, uint32_t kb, const double* __restrict__ u,
                                                   const double* __restrict__ A64, double sc, f2 t, float qd,
                                                   float qu, unsigned& recomputed, bool keep_fixed) {
    const int lane = threadIdx.x & 31;
    const double td = static_cast<double>(t.h) + static_cast<double>(t.l);
    while (__any_sync(FULL, amb != 0u)) {
        const int src = __ffs(__ballot_sync(FULL, amb != 0u)) - 1;
        const int bsel = __shfl_sync(FULL, __ffs(amb) - 1, src);
        const int ms = bsel >> 3, mr = bsel & 7;
        const double c = exact_coef(u, src & 7, (src >> 3) + 4 * ms, mr, A64, sc);
        ++recomputed;
        if (lane == src) {
            const bool keep = keep_fixed ? ((kb >> bsel) & 1u) != 0u : c * c >= td;
            float v = static_cast<float>(c);
            if (keep) v = static_cast<float>(rint(c * static_cast<double>(qd))) * qu;  // ties to even; exact
            buf[lane * 17 + bsel] = v;
            kb = keep ? (kb | (1u << bsel)) : (kb & ~(1u << bsel));
            amb &= ~(1u << bsel);
        }
    }
    __syncwarp();
    return kb;
}

// Cumulative-energy selection of an element that the fast path leaves open (a rare path; inlined,
// so that its call does not make the common path save registers around it): the modes kept are those whose energy is at least T, the smallest energy
// value v with sum_{a^2 <= v} a^2 > t.  FP64 mode recomputes the element's coefficients
// a' = 2^-ke A x A x A u in hardware FP64 from its doubles (reread from L2); the FP32 form
// takes its FP32 coefficients, passed at buf[lane * 17 + 8 s + r], as they are (their
// squares are exact in FP64).  The energies become 64-bit fixed-point keys floor(a^2 2^K)
// with t 2^K in [2^47, 2^48), so every sum is an exact integer sum whatever its order (the
// floors move a sum by at most 512 units, 4e-12 t), and a bisection on the key value finds
// T.  Returns the lane's keep bits (8 s + r); FP64 mode also leaves at buf[lane * 17 + b]
// each kept coefficient's code times 2^s (exact, so the quantisation reproduces the code of
// the FP64 value) and every other coefficient rounded to float.
template <bool DF>
__device__ __forceinline__ uint32_t cum_general(float* buf, const double* __restrict__ u, const double* __restrict__ A64,
                                             double sc, double td, float qd, float qu, unsigned& recomputed) {
    const int lane = threadIdx.x & 31, j = lane & 7, k0 = lane >> 3;
    double a[16];  // the lane's coefficients, b = 8 s + r: mode (p, q, r) = (j, k0 + 4 s, r)
    if constexpr (DF) {
        double* D = reinterpret_cast<double*>(buf);  // 512 doubles, the warp's buffer
        double x[8], y[8];
        __syncwarp();
#pragma unroll
        for (int s = 0; s < 2; ++s) {  // along i: pencils (k, j) = (k0 + 4 s, j) -> D[k][j][p]
            const double2* row = reinterpret_cast<const double2*>(u + (lane + 32 * s) * 8);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const double2 v = __ldg(row + c);
                x[2 * c] = v.x * sc;
                x[2 * c + 1] = v.y * sc;
            }
#pragma unroll
            for (int pp = 0; pp < 8; ++pp) {
                double acc = 0.0;
#pragma unroll
                for (int i = 0; i < 8; ++i) acc = fma(A64[pp * 8 + i], x[i], acc);
                y[pp] = acc;
            }
#pragma unroll
            for (int pp = 0; pp < 8; ++pp) D[((k0 + 4 * s) * 8 + j) * 8 + pp] = y[pp];
        }
        __syncwarp();
        double z[2][8];
#pragma unroll
        for (int s = 0; s < 2; ++s) {  // along j: lane (k, p) = (k0 + 4 s, j) -> D[k][q][p]
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) x[jj] = D[((k0 + 4 * s) * 8 + jj) * 8 + j];
#pragma unroll
            for (int qq = 0; qq < 8; ++qq) {
                double acc = 0.0;
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) acc = fma(A64[qq * 8 + jj], x[jj], acc);
                z[s][qq] = acc;
            }
        }
        __syncwarp();
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int qq = 0; qq < 8; ++qq) D[((k0 + 4 * s) * 8 + qq) * 8 + j] = z[s][qq];
        __syncwarp();
#pragma unroll
        for (int s = 0; s < 2; ++s) {  // along k: lane (q, p) = (k0 + 4 s, j) -> coefficient r
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) x[kk] = D[(kk * 8 + k0 + 4 * s) * 8 + j];
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) {
                double acc = 0.0;
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) acc = fma(A64[rr * 8 + kk], x[kk], acc);
                a[8 * s + rr] = acc;
            }
        }
        __syncwarp();
        recomputed += 512;
    } else {
#pragma unroll
        for (int b = 0; b < 16; ++b) a[b] = static_cast<double>(buf[lane * 17 + b]);
    }
    // keys and budget: t 2^K in [2^47, 2^48); energies of 2^50 / 2^K >= 4 t and more are clamped
    // (always kept)
    int ex;
    frexp(td, &ex);  // td in [2^(ex - 1), 2^ex)
    const double sK = ldexp(1.0, 48 - ex);
    const unsigned long long tt = static_cast<unsigned long long>(td * sK);
    constexpr unsigned long long kClamp = 1ull << 50;
    unsigned long long key[16];
    unsigned long long own = 0ull;
#pragma unroll
    for (int b = 0; b < 16; ++b) {
        const double v = a[b] * a[b] * sK;
        key[b] = v >= static_cast<double>(kClamp) ? kClamp : static_cast<unsigned long long>(v);
        own += key[b];
    }
    uint32_t kb = 0;
    if (warp_sum_u62(own) > tt) {  // else every energy fits the budget: nothing kept
        unsigned long long lo = 1, hi = kClamp;  // smallest v with sum_{key <= v} key > tt
        while (lo < hi) {
            const unsigned long long mid = lo + (hi - lo) / 2;
            unsigned long long sm = 0ull;
#pragma unroll
            for (int b = 0; b < 16; ++b) sm += key[b] <= mid ? key[b] : 0ull;
            if (warp_sum_u62(sm) > tt) hi = mid;
            else lo = mid + 1;
        }
#pragma unroll
        for (int b = 0; b < 16; ++b) kb |= (key[b] >= lo ? 1u : 0u) << b;
    }
    if constexpr (DF) {
#pragma unroll
        for (int b = 0; b < 16; ++b)
            buf[lane * 17 + b] = ((kb >> b) & 1u) ? static_cast<float>(rint(a[b] * static_cast<double>(qd))) * qu
                                                  : static_cast<float>(a[b]);
        __syncwarp();
    }
    return kb;
}

// 8-point even-odd folded inverse in FP32, both pencils packed (tables from the constant bank).
__device__ __forceinline__ void w_inv2(const float* __restrict__ Ph, const float2 (&x)[8], float2 (&y)[8]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 e = f2fma(f2dup(Ph[i * 8 + 6]), x[6], f2fma(f2dup(Ph[i * 8 + 4]), x[4],
                         f2fma(f2dup(Ph[i * 8 + 2]), x[2], f2mul(f2dup(Ph[i * 8]), x[0]))));
        const float2 o = f2fma(f2dup(Ph[i * 8 + 7]), x[7], f2fma(f2dup(Ph[i * 8 + 5]), x[5],
                         f2fma(f2dup(Ph[i * 8 + 3]), x[3], f2mul(f2dup(Ph[i * 8 + 1]), x[1]))));
        y[i] = f2add(e, o);
        y[7 - i] = f2sub(e, o);
    }
}

// Dense folded inverse in FP32 for an element that keeps many modes (rare, out of
// line): r (registers) -> k, q -> j, p -> i through the warp's buffer, the lane's two
// pencils packed.  Input: the kept values (code x 2^s, else 0) of the lane's
// coefficients (s, r) at buf[(lane + 32 s) * 9 + r]; result: its nodal pencils
// (k0 + 4s, j) at buf[(lane + 32 s) * 9 + i].
__device__ __noinline__ void dense_inverse_f32(float* buf, const float* Ph) {
    const int lane = threadIdx.x & 31, j = lane & 7, k0 = lane >> 3;
    float2 x[8], y[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) x[r] = make_float2(buf[lane * 9 + r], buf[(lane + 32) * 9 + r]);
    w_inv2(Ph, x, y);  // lane (q = k0 + 4s, p = j): values over k
    __syncwarp();
    {
        float4* d0 = reinterpret_cast<float4*>(buf + k0 * TSK + j * TSJ);
        float4* d1 = reinterpret_cast<float4*>(buf + (k0 + 4) * TSK + j * TSJ);
        d0[0] = make_float4(y[0].x, y[1].x, y[2].x, y[3].x);
        d0[1] = make_float4(y[4].x, y[5].x, y[6].x, y[7].x);
        d1[0] = make_float4(y[0].y, y[1].y, y[2].y, y[3].y);
        d1[1] = make_float4(y[4].y, y[5].y, y[6].y, y[7].y);
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 8; ++q)  // lane (k = k0 + 4s, p = j): values over q
        x[q] = make_float2(buf[q * TSK + j * TSJ + k0], buf[q * TSK + j * TSJ + k0 + 4]);
    w_inv2(Ph, x, y);
    __syncwarp();
    {
        float4* d0 = reinterpret_cast<float4*>(buf + k0 * TSK + j * TSJ);
        float4* d1 = reinterpret_cast<float4*>(buf + (k0 + 4) * TSK + j * TSJ);
        d0[0] = make_float4(y[0].x, y[1].x, y[2].x, y[3].x);
        d0[1] = make_float4(y[4].x, y[5].x, y[6].x, y[7].x);
        d1[0] = make_float4(y[0].y, y[1].y, y[2].y, y[3].y);
        d1[1] = make_float4(y[4].y, y[5].y, y[6].y, y[7].y);
    }
    __syncwarp();
#pragma unroll
    for (int pp = 0; pp < 8; ++pp)  // lane (k = k0 + 4s, j): values over p
        x[pp] = make_float2(buf[k0 * TSK + pp * TSJ + j], buf[(k0 + 4) * TSK + pp * TSJ + j]);
    w_inv2(Ph, x, y);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        buf[lane * 9 + i] = y[i].x;
        buf[(lane + 32) * 9 + i] = y[i].y;
    }
    __syncwarp();
}

// 8-point even-odd folded inverse in float pairs, both pencils packed (tables from the
// constant bank): y[i] = sum_p Phi[i][p] x[p].
__device__ __forceinline__ void w_inv_df2(const float* __restrict__ Ph, const float* __restrict__ Pl,
                                          const p2 (&x)[8], p2 (&y)[8]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        p2 e = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)}, o = e;
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            const p2 c = {f2dup(Ph[i * 8 + p]), f2dup(Pl[i * 8 + p])};
            if ((p & 1) == 0) df_fma_acc2(e, c, x[p]);
            else df_fma_acc2(o, c, x[p]);
        }
        e = df_norm2(e);
        o = df_norm2(o);
        y[i] = df_add2(e, o);
        y[7 - i] = df_sub2(e, o);
    }
}

// Dense folded inverse in float pairs for an element that keeps many modes (a
// rare path, kept out of line so that its registers do not weigh on the
// common one): r (registers) -> k, q -> j, p -> i through the warp's buffer,
// the lane's two pencils packed.  Input as dense_inverse_f32 (floats); result:
// the lane's nodal pencils (k0 + 4s, j) at buf[(lane + 32 s) * 9 + i] (pairs).
__device__ __noinline__ void dense_inverse_pairs(float2* buf, const float* Ph, const float* Pl) {
    const int lane = threadIdx.x & 31, j = lane & 7, k0 = lane >> 3;
    const float* vin = reinterpret_cast<const float*>(buf);
    p2 x[8], y[8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
        x[r] = {make_float2(vin[lane * 9 + r], vin[(lane + 32) * 9 + r]), make_float2(0.0f, 0.0f)};
    w_inv_df2(Ph, Pl, x, y);  // lane (q = k0 + 4s, p = j): values over k
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
            buf[(k0 + 4 * s) * TSK2 + j * TSJ2 + kk] = s ? make_float2(y[kk].h.y, y[kk].l.y) : make_float2(y[kk].h.x, y[kk].l.x);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 8; ++q) {  // lane (k = k0 + 4s, p = j): values over q
        const float2 v0 = buf[q * TSK2 + j * TSJ2 + k0], v1 = buf[q * TSK2 + j * TSJ2 + k0 + 4];
        x[q] = {make_float2(v0.x, v1.x), make_float2(v0.y, v1.y)};
    }
    w_inv_df2(Ph, Pl, x, y);
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
            buf[(k0 + 4 * s) * TSK2 + j * TSJ2 + jj] = s ? make_float2(y[jj].h.y, y[jj].l.y) : make_float2(y[jj].h.x, y[jj].l.x);
    __syncwarp();
#pragma unroll
    for (int pp = 0; pp < 8; ++pp) {  // lane (k = k0 + 4s, j): values over p
        const float2 v0 = buf[k0 * TSK2 + pp * TSJ2 + j], v1 = buf[(k0 + 4) * TSK2 + pp * TSJ2 + j];
        x[pp] = {make_float2(v0.x, v1.x), make_float2(v0.y, v1.y)};
    }
    w_inv_df2(Ph, Pl, x, y);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        buf[lane * 9 + i] = make_float2(y[i].h.x, y[i].l.x);
        buf[(lane + 32) * 9 + i] = make_float2(y[i].h.y, y[i].l.y);
    }
    __syncwarp();
}

// BATCH = false: one reduction, parameters and tensor maps in A.  BATCH = true: the
// work queue q of several lx = 8 reductions (each with its own descriptor, payload
// and scratch; their tensor maps in global memory at q.tmaps, field_base order).
// CTAs per SM the register budget aims at (measured): FP64 mode 4 (128 registers; the low words
// of u parked in shared memory keep it nearly free of spills), the FP32 form 6 (80) and 5 (96, no
// spills) with the cumulative variant.
template <int MODE, bool BATCH, bool CUM = false>
__global__ void __launch_bounds__(WPB * 32, MODE ? 4 : (CUM ? 5 : 6))
    reduce_warp_kernel(const __grid_constant__ WArgs A, const BatchQueue q) {
    constexpr bool DF = MODE != 0;
    using SM = WSmem<DF>;
    extern __shared__ uint8_t smem_raw[];
    // the stages start 512-byte aligned: the 64-byte swizzle permutes 16-byte chunks by address bits 7-8
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 511) & ~uintptr_t(511));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

    float* sPTh = reinterpret_cast<float*>(smem + SM::off_tab);  // [p][i] = Phi[i][p]
    float* sPTl = sPTh + 64;
    float2* sPT2h = reinterpret_cast<float2*>(smem + SM::off_dup);  // [p][i] = (Phi[i][p], Phi[i][p])
    float2* sPT2l = sPT2h + 64;                                        // FP64 mode: low words
    for (int t = threadIdx.x; t < 64; t += WPB * 32) {
        const int i = t >> 3, c = t & 7;  // Ph[t] = Phi[i][c]
        sPTh[c * 8 + i] = A.tab.Ph[t];
        sPTl[c * 8 + i] = A.tab.Pl[t];
        sPT2h[c * 8 + i] = f2dup(A.tab.Ph[t]);
        if constexpr (DF) sPT2l[c * 8 + i] = f2dup(A.tab.Pl[t]);
    }
    // quadrature weight products w_i w_j w_k of point i of pencils P = lane and lane + 32 (P = j + 8k):
    // FP64 mode [i][lane] = (hi0, hi1, lo0, lo1); the FP32 form forms its error sums as
    // sum_i w_i (w_j w_k d_i^2) with the w_j w_k of its two pencils in a register pair
    for (int t = threadIdx.x; DF && t < 512; t += WPB * 32) {
        const int i = t >> 6, P = t & 63, jj = P & 7, kk = P >> 3;
        const f2 w3 = df_mul({A.tab.wh[i], A.tab.wl[i]},
                             df_mul({A.tab.wh[jj], A.tab.wl[jj]}, {A.tab.wh[kk], A.tab.wl[kk]}));
        float* wt = reinterpret_cast<float*>(smem + SM::off_wq) + (i * 32 + (P & 31)) * 4;
        wt[P >> 5] = w3.h;
        wt[2 + (P >> 5)] = w3.l;
    }
    uint8_t* wb = smem + SM::off_warp + wid * SM::wbytes;
    uint8_t* stage = smem + wid * SM::stage;
    WStash* s_res = reinterpret_cast<WStash*>(smem + SM::off_res);
    float* tb = reinterpret_cast<float*>(wb + SM::o_tb);
    float2* tb2 = reinterpret_cast<float2*>(wb + SM::o_tb);
    uint32_t* smask = reinterpret_cast<uint32_t*>(wb + SM::o_mask);
    int2* skl = reinterpret_cast<int2*>(wb + SM::o_kl);
    uint64_t* bar = reinterpret_cast<uint64_t*>(wb + SM::o_bar);
    float2* sul = reinterpret_cast<float2*>(wb + SM::o_ul);  // FP64 mode only
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    // this lane's pencils: (k, j) = (k0 + 4s, j) in nodal phases, (k0 + 4s, j) -> (q, p) in modal ones
    const int j = lane & 7, k0 = lane >> 3;
    const int sw = (lane >> 1) & 3;  // 64-byte swizzle of rows lane and lane + 32
    // FP32 form: w_j w_k of this lane's pencils (k0, j) and (k0 + 4, j)
    const float2 wjk = make_float2(df_mul({A.tab.wh[j], A.tab.wl[j]}, {A.tab.wh[k0], A.tab.wl[k0]}).h,
                                   df_mul({A.tab.wh[j], A.tab.wl[j]}, {A.tab.wh[k0 + 4], A.tab.wl[k0 + 4]}).h);
    const float4* sWq4 = reinterpret_cast<const float4*>(smem + SM::off_wq);

    const uint32_t total_tiles = BATCH ? static_cast<uint32_t>(q.total_tiles) : A.total_tiles;
    unsigned* counter = BATCH ? q.counter : &A.p.ctl->tile_counter;
    const CUtensorMap* qmaps = reinterpret_cast<const CUtensorMap*>(q.tmaps);
    // this CTA's staging (a tile's codes are placed one tile later): codes [2 tile parities][warp]
    // [kWarpArena], within-tile prefixes [2][kWarpTile + 1], arena offsets [2][kWarpTile]; a batched
    // launch's items share it
    uint8_t* stage_cta = reinterpret_cast<uint8_t*>(BATCH ? q.items[0].code_stage : A.p.code_stage) +
                         static_cast<uint64_t>(blockIdx.x) * kWarpStageBytes;
    if (!bchk(static_cast<int>(blockIdx.x) < (BATCH ? q.items[0].stage_ctas : A.p.stage_ctas),
              BATCH ? &q.items[0].ctl->status : &A.p.ctl->status))
        return;  // (before any barrier or copy) a grid larger than the code staging
    int16_t* stage_codes = reinterpret_cast<int16_t*>(stage_cta);
    uint32_t* stage_pre = reinterpret_cast<uint32_t*>(stage_cta + 2ull * WPB * kWarpArena * 2);
    uint32_t* stage_off = stage_pre + 2 * (kWarpTile + 1);
    constexpr uint32_t kDirect = 0xffffffffu;  // arena offset of an element written directly

    // tiles: kWarpTile consecutive elements of one field; warp w takes elements w, w + 4, ...
    __shared__ uint32_t s_tile[2];  // current tile; the next one, claimed when the current one is computed
    __shared__ uint32_t s_titem[2], s_tloc[2];    // their item and tile index within the item (BATCH)
    __shared__ LaunchParams s_par[BATCH ? 2 : 1];  // BATCH: descriptors of the current and previous tile
    // item and local tile of a claimed global tile (thread 0)
    auto resolve = [&](uint32_t g, int slot) {
        uint32_t item = 0, loc = g;
        if (BATCH && g < total_tiles) {  // last item whose first tile is <= g
            int lo = 0, hi = q.n_items - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) / 2;
                if (q.tile_base[mid] <= g) lo = mid; else hi = mid - 1;
            }
            item = static_cast<uint32_t>(lo);
            loc = g - static_cast<uint32_t>(q.tile_base[lo]);
        }
        s_titem[slot] = item;
        s_tloc[slot] = loc;
    };
    __shared__ uint32_t s_cnt[kWarpTile];  // tile tag << 16 | code count; tag 0xffff: nothing yet
    __shared__ unsigned long long s_excl;
    __shared__ unsigned long long s_peek;  // a tile's exclusive prefix for directly written codes
    __shared__ uint32_t s_peek_tag;        // that tile + 1 (0: none)
    __shared__ double s_wpart[WPB][4];  // per-warp partials of the tile
    __shared__ int s_abort;
    if (threadIdx.x == 0) {
        s_tile[0] = atomicAdd(counter, 1u);
        resolve(s_tile[0], 0);
        s_abort = 0;
        s_peek_tag = 0;
    }
    for (int i = threadIdx.x; i < kWarpTile; i += WPB * 32) s_cnt[i] = 0xffff0000u;
    __syncthreads();
    // field, first element and element count of local tile tt of an item with tpf tiles per field
    auto geom = [&](uint32_t tt, uint32_t tpf_, uint32_t E_, uint32_t& f, uint32_t& e0, int& nh) {
        f = tt / tpf_;
        e0 = (tt - f * tpf_) * kWarpTile;
        nh = static_cast<int>(min(static_cast<uint32_t>(kWarpTile), E_ - e0));
    };
    auto issue = [&](const CUtensorMap* tm, uint32_t e) {  // lane 0: element block e of map tm into the stage
        tma_load_2d(stage, tm, 0, static_cast<int>(e * WNP), bar, SM::stage);
    };
    uint32_t parity = 0;
    uint32_t tag = 0;       // tags the counts of the current tile (0 .. 0xfffe, then wraps)
    bool inflight = false;  // a block is on its way into this warp's stage
    unsigned recomputed = 0;
    uint32_t t_prev = 0xffffffffu;  // this CTA's previous tile (local index), whose codes are still staged
    int nh_prev = 0, par = 0;       // its element count; staging parity of the current tile
    uint32_t tot_prev = 0;          // warp 0: its code count

    // Copy the staged codes of a tile (staging parity pp, nhp elements) to code_base + 2 (excl + prefix).
    auto place_codes = [&](const LaunchParams& p, int pp, int nhp, uint64_t excl) {
        unsigned* status = &p.ctl->status;
        const uint32_t* pre = stage_pre + pp * (kWarpTile + 1);
        const int16_t* arena = stage_codes + (pp * WPB + wid) * kWarpArena;
        // lane L: element wid + WPB L, one of the warp's own (its codes are in this warp's arena),
        // so the prefixes and offsets of all 32 elements are fetched at once and their (few) codes
        // are copied side by side
        const int il = wid + WPB * lane;
        uint32_t b = 0, n = 0, off = kDirect;
        if (il < nhp) {
            b = pre[il];
            n = pre[il + 1] - b;
            off = stage_off[pp * kWarpTile + il];
        }
        const uint64_t gbyte = p.code_base + 2ull * (excl + b);
        bool copy = off != kDirect && n > 0;  // (off == kDirect: written directly)
        if (copy && gbyte + 2ull * n > p.payload_cap) {
            atomicOr(status, static_cast<unsigned>(SEMR_STATUS_OVERFLOW));
            copy = false;
        }
        copy = copy && bchk(off + n <= static_cast<uint32_t>(kWarpArena) && gbyte >= p.code_base, status);
        if (copy && n <= 32u) {
            int16_t* dst = reinterpret_cast<int16_t*>(p.payload + gbyte);
            const int16_t* src = arena + off;
            for (uint32_t k = 0; k < n; ++k) dst[k] = src[k];
        }
        // elements with more codes: the whole warp copies each
        for (uint32_t big = __ballot_sync(FULL, copy && n > 32u); big; big &= big - 1) {
            const int src_lane = __ffs(big) - 1;
            const uint32_t nb = __shfl_sync(FULL, n, src_lane), ob = __shfl_sync(FULL, off, src_lane);
            int16_t* dst = reinterpret_cast<int16_t*>(p.payload + __shfl_sync(FULL, gbyte, src_lane));
            for (uint32_t k = lane; k < nb; k += 32) dst[k] = arena[ob + k];
        }
    };
    for (;;) {
    // Tiles are claimed only once the previous one is computed, so they start in about
    // the order of their claims and a look-back never waits for a tile not yet begun.
    if (s_tile[0] >= total_tiles) break;
    const uint32_t gtile = s_tile[0];
    const uint32_t item = s_titem[0], tcur = s_tloc[0];  // tcur: the tile's index within its item
    if constexpr (BATCH) {  // the item's descriptor into this tile's slot (the other holds the previous one's)
        __syncthreads();  // the slot's last reader (the placement of two tiles ago) is done
        constexpr int PW = sizeof(LaunchParams) / 4;
        static_assert(sizeof(LaunchParams) % 4 == 0, "descriptor copy by words");
        for (int i = threadIdx.x; i < PW; i += WPB * 32)
            reinterpret_cast<int*>(&s_par[par])[i] = reinterpret_cast<const int*>(&q.items[item])[i];
        __syncthreads();
    }
    const LaunchParams& p = BATCH ? s_par[par] : A.p;
    const LaunchParams& pprev = BATCH ? s_par[par ^ 1] : A.p;
    const uint32_t E = static_cast<uint32_t>(p.n_elem), tpf = static_cast<uint32_t>(p.tiles_per_field);
    const CUtensorMap* tmaps = BATCH ? qmaps + q.field_base[item] : A.tm;
    unsigned* status = &p.ctl->status;
    float tau_h = A.tau_h, tau_l = A.tau_l;
    if constexpr (BATCH) {
        tau_h = static_cast<float>(p.tau);
        tau_l = static_cast<float>(p.tau - static_cast<double>(tau_h));
    }
    uint32_t f, e0;
    int nh;
    geom(tcur, tpf, E, f, e0, nh);
    int16_t* arena = stage_codes + (par * WPB + wid) * kWarpArena;  // this warp's codes of the tile
    uint32_t atop = 0;                                             // its fill (warp-uniform)
    for (int il = wid; il < nh; il += WPB) {
        const uint32_t e = e0 + static_cast<uint32_t>(il);
        if (!inflight && lane == 0) issue(&tmaps[f], e);
        if (!mbar_wait_bounded(bar, parity)) {
            if (lane == 0) {
                atomicOr(status, static_cast<unsigned>(SEMR_STATUS_TIMEOUT));
                s_abort = 1;
            }
            drain_stage(bar, parity, status);  // the copy may still land: wait once more, bounded
            inflight = false;
            break;
        }
        parity ^= 1u;
        inflight = false;

        // ---- the element's largest high word of |u| (a first pass over the stage's high words)
        // (the lane's 16 doubles stay in registers for the split below)
        uint32_t hm = 0;
        uint4 raw[8];  // pencil lane + 32 (c >> 2), doubles 2 (c & 3) and 2 (c & 3) + 1
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            raw[c] = *reinterpret_cast<const uint4*>(stage + (lane + 32 * (c >> 2)) * 64 + (((c & 3) ^ sw) << 4));
            hm = max(hm, max(raw[c].y & 0x7fffffffu, raw[c].w & 0x7fffffffu));
        }
        const uint32_t hmax0 = __reduce_max_sync(FULL, hm);
        const bool bad = __any_sync(FULL, hm >= (static_cast<uint32_t>(1023 + 500) << 20));
        const bool tiny = __all_sync(FULL, hm < 0x00100000u);
        // exact power-of-two prescale: the element is read as u 2^-ke with ke the binary exponent
        // of its largest |u|, so every value formed below lies near 1 whatever the field's units
        // (masks and codes do not change under it; steps and norms are scaled back exactly).
        // NaN, infinity or |u| >= 2^500 (energies beyond FP64): flagged, keeps nothing; zeros and
        // subnormals only (|u| < 2^-1022): a zero block, keeps nothing
        const int bias = 0x38000000 + ((hmax0 < 0x00100000u ? 0 : min(static_cast<int>(hmax0 >> 20) - 1023, 1023)) << 20);
        if (lane == 0) {  // the element's stash entry keeps these (read back below, not held in registers)
            s_res[il].ke = (bias - 0x38000000) >> 20;
            s_res[il].hmax = hmax0;
        }
        // ---- the lane's two pencils, split into floats with integer instructions
        float2 uh[8], ul[8];  // (pencil lane, pencil lane + 32) at point i
#pragma unroll
        for (int pen = 0; pen < 2; ++pen) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint4 v = raw[4 * pen + c];
                const uint32_t lo[2] = {v.x, v.z}, hi[2] = {v.y, v.w};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int i = 2 * c + h;
                    float vh_, vl_ = 0.0f;
                    if constexpr (DF) w_split(lo[h], hi[h], bias, vh_, vl_);
                    else vh_ = w_d2f_rz(lo[h], hi[h], bias);
                    if (pen == 0) {
                        uh[i].x = vh_;
                        ul[i].x = vl_;
                    } else {
                        uh[i].y = vh_;
                        ul[i].y = vl_;
                    }
                }
            }
        }
        // ---- element energy S, FP64 mode: sum w u^2 at the nodes in pairs (Parseval's identity in
        // nodal form), right after the split; the low words then wait in the warp's slots until the
        // reconstruction starts from u (their registers are free in between)
        f2 S = {0.0f, 0.0f};
        if constexpr (DF) {
            p2 sp = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float4 w = sWq4[i * 32 + lane];
                const float2 ph = f2mul(uh[i], uh[i]);
                const float2 pl = f2fma(uh[i], f2add(ul[i], ul[i]), f2fma(uh[i], uh[i], f2neg(ph)));
                df_fma_acc2(sp, {make_float2(w.x, w.y), make_float2(w.z, w.w)}, {ph, pl});
            }
            sp = df_norm2(sp);
            S = warp_sum_pair(df_add({sp.h.x, sp.l.x}, {sp.h.y, sp.l.y}));
#pragma unroll
            for (int i = 0; i < 8; ++i) sul[i * 32 + lane] = ul[i];
        }
        // once every lane has consumed its loads, the stage may be refilled with this warp's
        // next element (an exact recomputation below rereads the block from global memory)
        __syncwarp();
        if (il + WPB < nh) {
            if (lane == 0) {
                fence_proxy_async();
                issue(&tmaps[f], e + WPB);
            }
            inflight = true;
        }

        // ---- forward transform (FP32, both pencils packed): i in registers, then j and k through
        // the warp's buffer.  Layout A [k0][j][p][s] (plane 176, row 20 floats) lets a lane read its
        // two values with one 8-byte load; layout B [k][p][q'] (plane 96, row 12) with the columns
        // in the order q' = (q & 3) 2 + (q >> 2) does the same for the last contraction.  Both are
        // free of bank conflicts for the 16-byte stores and 8-byte loads of a warp.
        float2 a2[8];  // coefficient r of modal pencils (q = k0 + 4s, p = j): mode lane + 32 s + 64 r
        {
            float2 y[8];
            w_fwd2(A.tab.A2, uh, y);
            float4* d = reinterpret_cast<float4*>(tb + k0 * 176 + j * 20);
#pragma unroll
            for (int c = 0; c < 4; ++c) d[c] = make_float4(y[2 * c].x, y[2 * c].y, y[2 * c + 1].x, y[2 * c + 1].y);
            __syncwarp();
            float2 x[8];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) x[jj] = *reinterpret_cast<const float2*>(tb + k0 * 176 + jj * 20 + 2 * j);
            w_fwd2(A.tab.A2, x, y);  // y[q] of pencils (k0, p = j) and (k0 + 4, p = j)
            __syncwarp();
            float4* d0 = reinterpret_cast<float4*>(tb + k0 * 96 + j * 12);
            float4* d1 = reinterpret_cast<float4*>(tb + (k0 + 4) * 96 + j * 12);
            d0[0] = make_float4(y[0].x, y[4].x, y[1].x, y[5].x);
            d0[1] = make_float4(y[2].x, y[6].x, y[3].x, y[7].x);
            d1[0] = make_float4(y[0].y, y[4].y, y[1].y, y[5].y);
            d1[1] = make_float4(y[2].y, y[6].y, y[3].y, y[7].y);
            __syncwarp();
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) x[kk] = *reinterpret_cast<const float2*>(tb + kk * 96 + j * 12 + 2 * k0);
            w_fwd2(A.tab.A2, x, a2);
        }

        // ---- element energy S, FP32 form: sum a^2 of the coefficients (FP64 mode formed it above)
        if constexpr (!DF) {
            float2 sp = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int r = 0; r < 8; ++r) sp = f2fma(a2[r], a2[r], sp);
            S = {warp_sum_f(sp.x + sp.y), 0.0f};
        }

        // ---- per element (warp-uniform): t = tau S, step s_e = floor((ex - 1) / 2) for
        // t = mu 2^ex, and g = the smallest float with g^2 >= t.  All of it for the prescaled
        // block: t' = t 2^-2ke, so ex = ex' + 2 ke and s_e = s' + ke with s' = floor((ex' - 1) / 2);
        // the codes rint(a' 2^-s') equal rint(a 2^-s_e)
        int emode = 0;  // 0: keep none, 1: threshold
        int step = INT16_MIN, sps = 0;  // s_e and s'
        f2 t = {0.0f, 0.0f};
        float g = 0.0f;
        const uint32_t hmax = s_res[il].hmax;
        const int ke = s_res[il].ke;
        if (bad || !isfinite(S.h)) {
            if (lane == 0) atomicOr(status, static_cast<unsigned>(SEMR_STATUS_NONFINITE));
        } else if (tiny) {  // zeros and subnormals only: keeps nothing, norms 0
            if (lane == 0 && hmax != 0u) atomicOr(status, static_cast<unsigned>(SEMR_STATUS_TINY));
        } else {
            // S' >= min w_i w_j w_k > 4e-5 (|u'| reaches 1) and 3.7e-9 < tau <= 2^64 (int16 codes),
            // so t' is a normal float
            t = df_norm(df_mul({tau_h, tau_l}, S));
            const uint32_t tb_ = __float_as_uint(t.h);
            int exs = static_cast<int>(tb_ >> 23) - 126;
            if ((tb_ & 0x7fffffu) == 0u && t.l < 0.0f) --exs;  // t just below a power of two
            const int ex = exs + 2 * ke;
            if (ex > 1024) {  // t = tau S_e overflows FP64
                if (lane == 0) atomicOr(status, static_cast<unsigned>(SEMR_STATUS_NONFINITE));
            } else if (ex >= -1021) {  // t >= 2^-1022, the smallest normal double
                sps = (exs - 1) >> 1;
                step = sps + ke;
                emode = 1;
                asm("sqrt.approx.f32 %0, %1;" : "=f"(g) : "f"(t.h));
#pragma unroll 1
                for (int it = 0; it < 4 && !sq_ge(g, t); ++it) g = __uint_as_float(__float_as_uint(g) + 1u);
#pragma unroll 1
                for (int it = 0; it < 4; ++it) {
                    const float pr = __uint_as_float(__float_as_uint(g) - 1u);
                    if (sq_ge(pr, t)) g = pr; else break;
                }
            }
        }
        // t' in [1e-13, 2^70] keeps s' in [-22, 35]: 2^-s' and 2^s' are normal floats (exact scalings)
        const float qd = pow2f(-sps), qu = pow2f(sps);

        // ---- keep decisions; FP64 mode recomputes exactly what FP32 cannot settle
        uint32_t kb = 0;  // keep bit (8 s + r)
        // FP64 mode: the rounding decisions of the lane's kept coefficients (a few per element,
        // so a loop over the lane's keep bits), with Mq the bound in units of the step
        auto screen_roundings = [&](uint32_t keep, float Mq) -> uint32_t {
            uint32_t amb = 0;
            for (uint32_t kk = keep; kk; kk &= kk - 1) {
                const int b = __ffs(kk) - 1;
                const float y = fabsf(pick(a2, 2 * (b & 7) + (b >> 3))) * qd;  // word s + 2 r of bit 8 s + r
                if (fabsf((y - floorf(y)) - 0.5f) <= Mq + y * 1.2e-7f) amb |= 1u << b;
            }
            return amb;
        };
        if constexpr (CUM) {
            if (emode == 1) {
                // cumulative-energy truncation: keep the modes whose energy is at least T, the
                // smallest energy value v with sum_{a^2 <= v} a^2 > t.  Every mode with a^2 > t is
                // kept (the dropped ones fit the budget t); of the rest, extract the largest |a| one
                // at a time, subtracting its square from R, the sum of the squares not extracted
                // yet, until R <= t: the last one extracted is the smallest kept (ties with it are
                // kept too).  FP64 mode takes the result only where the FP32 coefficients' bound M
                // settles it -- t - R, R + (v - M)^2 - t and the gap between v and the largest
                // coefficient left all clear of B = 2 M sum_{left} |a| + n M^2 plus the FP32 sums'
                // rounding -- else (and beyond kCumIters extractions) the general path decides.
                constexpr int kCumIters = 48;
                float M = 0.0f, gb;  // gb: |a| >= gb surely has a^2 > t
                if constexpr (DF) {
                    constexpr float kMarg = (3.0f * (4 + 2) + 2.0f) * 5.9604645e-8f * 2.8285f * 2.0f;
                    const float umax_e = __uint_as_float(0x3f800000u | ((hmax & 0xfffffu) << 3));
                    M = kMarg * umax_e * 1.000002f;
                    gb = g + (M + g * 2.4e-7f);
                } else {
                    gb = __uint_as_float(__float_as_uint(g) + 1u);  // |a| > g
                }
                auto absbits = [&](int b) -> uint32_t {
                    return __float_as_uint(b & 8 ? a2[b & 7].y : a2[b & 7].x) & 0x7fffffffu;
                };
                uint32_t rem = 0;  // the lane's coefficients below gb, not extracted yet
                float rs = 0.0f, sa = 0.0f;
#pragma unroll
                for (int b = 0; b < 16; ++b) {
                    const float x = __uint_as_float(absbits(b));
                    const bool low = x < gb;
                    rem |= (low ? 1u : 0u) << b;
                    rs = low ? fmaf(x, x, rs) : rs;
                    sa = low ? sa + x : sa;
                }
                float R = warp_sum_f(rs);
                float sabs = warp_sum_f(sa);
                const float R0 = R;
                int nrem = static_cast<int>(__reduce_add_sync(FULL, static_cast<unsigned>(__popc(rem))));
                int it = 0;
                float v = 0.0f;  // |a| of the last one extracted
                uint32_t wm = 0;
                bool done = R <= t.h, open = false;
                for (;;) {
                    uint32_t mk = 0;  // the largest coefficient left (the next to extract)
#pragma unroll
                    for (int b = 0; b < 16; ++b) mk = ((rem >> b) & 1u) ? max(mk, absbits(b)) : mk;
                    wm = __reduce_max_sync(FULL, mk);
                    if (done) break;
                    if (it == kCumIters || wm == 0u) {  // (only zeros left with R > t: not settled)
                        open = true;
                        break;
                    }
                    if (lane == __ffs(__ballot_sync(FULL, mk == wm)) - 1) {  // one holder of it
                        uint32_t hit = 0;
#pragma unroll
                        for (int b = 0; b < 16; ++b) hit |= (((rem >> b) & 1u) && absbits(b) == wm ? 1u : 0u) << b;
                        rem &= ~(hit & (0u - hit));
                    }
                    v = __uint_as_float(wm);
                    R = fmaf(-v, v, R);
                    sabs -= v;
                    --nrem;
                    ++it;
                    done = R <= t.h;
                }
                bool settled = !open;
                if constexpr (DF) {
                    if (settled) {
                        // the smallest kept coefficient: the last extracted, else the smallest above gb
                        float vk = v;
                        if (it == 0) {
                            uint32_t mn = 0x7f000000u;  // (2^127: nothing above gb)
#pragma unroll
                            for (int b = 0; b < 16; ++b) mn = ((rem >> b) & 1u) ? mn : min(mn, absbits(b));
                            vk = __uint_as_float(__reduce_min_sync(FULL, mn));
                        }
                        const float wn = __uint_as_float(wm);  // the largest coefficient not kept
                        const float rho = R0 * (6e-5f + 1.2e-7f * static_cast<float>(it)) + 2.4e-7f * t.h;
                        const float B = 2.0f * M * sabs * 1.0001f + static_cast<float>(nrem) * M * M + rho;
                        const float d1 = t.h - R;  // >= 0
                        settled = d1 * 0.999999f > B;
                        if (vk < 0x1p126f) {  // something is kept
                            const float lv = fmaxf(vk - M, 0.0f);
                            settled = settled && (lv * lv * 0.999999f - d1 * 1.000001f) > B &&
                                      (vk - wn) > 2.0f * M * 1.000001f + vk * 1.2e-7f;
                        }
                    }
                }
                bool exactv = false;  // FP64 mode: a2 holds exact codes x 2^s where kept
                if (!settled) {
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        tb[lane * 17 + r] = a2[r].x;
                        tb[lane * 17 + 8 + r] = a2[r].y;
                    }
                    kb = cum_general<DF>(tb, p.fields[f] + static_cast<uint64_t>(e) * WN3, A.tab.A64, pow2d(-ke),
                                         static_cast<double>(t.h) + static_cast<double>(t.l), qd, qu, recomputed);
                    if constexpr (DF) {
#pragma unroll
                        for (int r = 0; r < 8; ++r) a2[r] = make_float2(tb[lane * 17 + r], tb[lane * 17 + 8 + r]);
                        exactv = true;
                    }
                    __syncwarp();
                } else {
                    // kept: everything at or above gb and every extracted coefficient, i.e. |a| >= v
                    // (ties included), or |a| >= gb when nothing was extracted
                    const uint32_t vb = __float_as_uint(it ? v : gb);
#pragma unroll
                    for (int b = 0; b < 16; ++b) kb |= (absbits(b) >= vb ? 1u : 0u) << b;
                }
                if constexpr (DF) {  // the rounding decisions of the kept coefficients
                    if (!exactv) {
                        const uint32_t amb = screen_roundings(kb, M * qd * 1.000001f);
                        if (__any_sync(FULL, amb != 0u)) {
#pragma unroll
                            for (int r = 0; r < 8; ++r) {
                                tb[lane * 17 + r] = a2[r].x;
                                tb[lane * 17 + 8 + r] = a2[r].y;
                            }
                            kb = resolve_ambiguous(tb, amb, kb, p.fields[f] + static_cast<uint64_t>(e) * WN3,
                                                   A.tab.A64, pow2d(-ke), t, qd, qu, recomputed, true);
#pragma unroll
                            for (int r = 0; r < 8; ++r) a2[r] = make_float2(tb[lane * 17 + r], tb[lane * 17 + 8 + r]);
                        }
                    }
                }
            }
        } else if (emode == 1) {
            if constexpr (DF) {
                // |a_fp32 - a| <= M: (H + 2) roundings per folded contraction (H = 4 terms, the fold,
                // the table), 3 contractions, 2 more for the input split; every row of A has
                // sum |A_pi| <= sqrt(2), so (|A|^3 |u|)_m <= 2^1.5 max|u|; a factor 2 of safety
                constexpr float kMarg = (3.0f * (4 + 2) + 2.0f) * 5.9604645e-8f * 2.8285f * 2.0f;
                // max |u 2^-ke| rounded toward zero to float: the top 20 mantissa bits of hmax, in [1, 2)
                const float umax_e = __uint_as_float(0x3f800000u | ((hmax & 0xfffffu) << 3));
                const float M = kMarg * umax_e * 1.000002f;
                const float Mg = M + g * 2.4e-7f;  // plus the float rounding of g +- M
                uint32_t amb = 0;
#pragma unroll
                for (int s = 0; s < 2; ++s)
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        const float aa = fabsf(s ? a2[r].y : a2[r].x);
                        const int b = 8 * s + r;
                        if (aa >= g + Mg) kb |= 1u << b;            // surely kept
                        else if (!(aa < g - Mg)) amb |= 1u << b;   // undecided
                    }
                amb |= screen_roundings(kb, Mg * qd);
                // exact (float-pair) coefficient of each ambiguous mode (rare): out of line, with
                // the lane's coefficients passed through the warp's transpose buffer (free here)
                if (__any_sync(FULL, amb != 0u)) {
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        tb[lane * 17 + r] = a2[r].x;
                        tb[lane * 17 + 8 + r] = a2[r].y;
                    }
                    kb = resolve_ambiguous(tb, amb, kb, p.fields[f] + static_cast<uint64_t>(e) * WN3, A.tab.A64,
                                           pow2d(-ke), t, qd, qu, recomputed, false);
#pragma unroll
                    for (int r = 0; r < 8; ++r) a2[r] = make_float2(tb[lane * 17 + r], tb[lane * 17 + 8 + r]);
                }
            }
        }

        // ---- mask words: the ballot over (slot s, row r) is word w = s + 2r (bit = lane).  Lane 0
        // stores the 16 words to shared memory (and the payload); lane w < 16 then reads word w, so
        // the count is one warp reduction and nzw (the words holding kept modes) one ballot.  The
        // FP32 form ballots its threshold test directly; FP64 mode ballots its settled keep bits
        uint8_t* fsec = p.payload + p.header_bytes + static_cast<uint64_t>(f) * p.fixed_bytes;
        // bounds build: the element, its field section and the section's layout within the payload
        const bool eok = bchk(f < static_cast<uint32_t>(p.n_fields) && e < E &&
                                  64ull * E + 2 * pad16(2ull * E) <= p.fixed_bytes &&
                                  p.header_bytes + (f + 1ull) * p.fixed_bytes <= p.code_base &&
                                  p.code_base <= p.payload_cap,
                              status);
        uint4* mdst = reinterpret_cast<uint4*>(fsec + static_cast<uint64_t>(e) * 64);
        uint32_t n_e = 0, nzw = 0;
        if constexpr (DF || CUM) {
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {  // words 4 q4 .. 4 q4 + 3
                uint32_t w4[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) w4[h] = __ballot_sync(FULL, (kb >> (8 * (h & 1) + 2 * q4 + (h >> 1))) & 1u);
                if (lane == 0) reinterpret_cast<uint4*>(smask)[q4] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
            }
            __syncwarp();
            const uint32_t mw = (lane < 16) ? smask[lane] : 0u;
            if (lane < 16 && eok) reinterpret_cast<uint32_t*>(mdst)[lane] = mw;
            n_e = __reduce_add_sync(FULL, static_cast<unsigned>(__popc(mw)));
            nzw = __ballot_sync(FULL, mw != 0u);
        } else {
            uint32_t wv[16];
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int s = 0; s < 2; ++s)  // keep iff |a| >= g, the exact float threshold
                    wv[s + 2 * r] = __ballot_sync(FULL, emode == 1 && fabsf(s ? a2[r].y : a2[r].x) >= g);
            if (lane == 0) {
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    const uint4 v = make_uint4(wv[4 * q4], wv[4 * q4 + 1], wv[4 * q4 + 2], wv[4 * q4 + 3]);
                    if (eok) mdst[q4] = v;
                    reinterpret_cast<uint4*>(smask)[q4] = v;
                }
            }
            __syncwarp();
            const uint32_t mw = (lane < 16) ? smask[lane] : 0u;
            n_e = __reduce_add_sync(FULL, static_cast<unsigned>(__popc(mw)));
            nzw = __ballot_sync(FULL, mw != 0u);
        }
        // payload: step and count (lane 0)
        const uint64_t mb = static_cast<uint64_t>(E) * 64;  // mask section (a multiple of 16)
        int16_t* sdst = reinterpret_cast<int16_t*>(fsec + mb);
        uint16_t* cdst = reinterpret_cast<uint16_t*>(fsec + mb + pad16(2ull * E));
        // the element's codes fit the warp's arena (else they are written directly)
        const bool staged = atop + n_e <= static_cast<uint32_t>(kWarpArena);
        if (lane == 0) {
            if (eok) {
                sdst[e] = static_cast<int16_t>(step);
                cdst[e] = static_cast<uint16_t>(n_e);
            }
            s_cnt[il] = (tag << 16) | n_e;
            stage_off[par * kWarpTile + il] = staged ? atop : kDirect;
        }
        if (e + 1 == E && lane < 16 && eok) {  // zero the padding after the step and count sections
            const uint64_t se = 2ull * E;
            if (se + lane < pad16(se)) {
                reinterpret_cast<uint8_t*>(sdst)[se + lane] = 0;
                reinterpret_cast<uint8_t*>(cdst)[se + lane] = 0;
            }
        }

        // ---- quantise: code = rint(a 2^-s), ties to even (exact: a 2^-s is a power-of-two scaling),
        // to the warp's arena, or straight to the payload when the arena is full
        int16_t* qdst = arena + atop;
        bool qwrite = true;
        if (!staged) {
            // the warp's arena is full (extreme inputs only): write the codes at their final place,
            // which needs the tile's exclusive prefix (computed once per tile) and the counts of the
            // tile's earlier elements; every such wait points to smaller element indices, so it ends
            uint64_t before;
            if (s_peek_tag == gtile + 1u) {
                before = s_peek;
            } else {
                before = lookback_peek(p.tile_state, tcur, status);
                if (lane == 0) {
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
            if (!qwrite && lane == 0) atomicOr(status, static_cast<unsigned>(SEMR_STATUS_OVERFLOW));
            qwrite = qwrite && bchk(gbyte >= p.code_base, status);
            qdst = reinterpret_cast<int16_t*>(p.payload + gbyte);
        }
        __syncwarp();
        {
            if constexpr (DF) {  // the lane's coefficients by word index w = s + 2r, in the warp's
                // transpose buffer (free here; rows of 20 floats, conflict-free 16-byte stores)
                float4* arow = reinterpret_cast<float4*>(tb + lane * 20);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    arow[q] = make_float4(a2[2 * q].x, a2[2 * q].y, a2[2 * q + 1].x, a2[2 * q + 1].y);
            }
            const uint32_t lt_mask = (1u << lane) - 1u;
            uint32_t run = 0;  // codes of the words before wi (the words come in increasing order)
            while (nzw) {
                const int wi = __ffs(nzw) - 1;
                nzw &= nzw - 1;
                const uint32_t wd = smask[wi];
                if ((wd >> lane) & 1u) {
                    const float a = DF ? tb[lane * 20 + wi] : pick(a2, wi);
                    const float c = (a * qd + 12582912.0f) - 12582912.0f;  // round half to even (|y| < 2^22)
                    const uint32_t rank = run + __popc(wd & lt_mask);
                    if (qwrite) qdst[rank] = static_cast<int16_t>(c);
                    if (rank < static_cast<uint32_t>(wsparse<DF>())) skl[rank] = make_int2(lane + 32 * wi, __float_as_int(c));
                }
                run += __popc(wd);
            }
        }
        if (staged) atop += n_e;
        __syncwarp();

        // ---- reconstruction of the lane's nodal pencils (both packed).  FP64 mode accumulates
        // d = u - u~ in pairs: the accumulators start at u and every kept mode is subtracted, so the
        // errors read d directly (a requested u~ is written as u - d in FP64 below); the FP32 form
        // accumulates u~
        float2 vh[8], vl[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            vh[i] = DF ? uh[i] : make_float2(0.0f, 0.0f);
            vl[i] = DF ? sul[i * 32 + lane] : make_float2(0.0f, 0.0f);
        }
        if (n_e <= static_cast<uint32_t>(wsparse<DF>())) {
            if constexpr (DF) {
                // d(i) = u(i) + sum over kept modes of B phi_p(x_i), B = -c 2^s phi_q(x_j) phi_r(x_k) per
                // pencil, both pencils packed.  Two passes over the kept list: the modes with p = 0
                // (phi_0 is constant along the pencil) give one pair per pencil added to every point;
                // each other mode adds B phi_p(x_i) at the eight points
                auto coef = [&](int2 kv) -> p2 {  // B of both pencils (k0, k0 + 4) as packed pairs
                    const int qq = (kv.x >> 3) & 7, rr = kv.x >> 6;
                    const float2 cs = f2dup(-(__int_as_float(kv.y) * qu));  // -c 2^s, exact
                    const float2 fjh = f2dup(sPTh[qq * 8 + j]), fjl = f2dup(sPTl[qq * 8 + j]);
                    const float2 frh = make_float2(sPTh[rr * 8 + k0], sPTh[rr * 8 + k0 + 4]);
                    const float2 frl = make_float2(sPTl[rr * 8 + k0], sPTl[rr * 8 + k0 + 4]);
                    const float2 ph = f2mul(fjh, frh);
                    const float2 pl = f2add(f2fma(fjh, frh, f2neg(ph)), f2fma(fjh, frl, f2mul(fjl, frh)));
                    const float2 bh = f2mul(ph, cs);
                    return {bh, f2fma(pl, cs, f2fma(ph, cs, f2neg(bh)))};
                };
                p2 c0 = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
                for (uint32_t tk = 0; tk < n_e; ++tk) {
                    const int2 kv = skl[tk];
                    if ((kv.x & 7) != 0) continue;
                    const p2 B = coef(kv);
                    const p2 sm = two_sum2(c0.h, B.h);
                    c0 = fast_two_sum2(sm.h, f2add(sm.l, f2add(c0.l, B.l)));
                }
                {  // times phi_0, the same at every point
                    const p2 ph0 = {f2dup(sPTh[0]), f2dup(sPTl[0])};
                    p2 v0 = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
                    df_fma_acc2(v0, c0, ph0);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const p2 sm = two_sum2(vh[i], v0.h);
                        vh[i] = sm.h;
                        vl[i] = f2add(vl[i], f2add(sm.l, v0.l));
                    }
                }
                for (uint32_t tk = 0; tk < n_e; ++tk) {
                    const int2 kv = skl[tk];
                    const int pp = kv.x & 7;
                    if (pp == 0) continue;
                    const p2 Bp = coef(kv);
                    const float4* ch4 = reinterpret_cast<const float4*>(sPT2h + pp * 8);
                    const float4* cl4 = reinterpret_cast<const float4*>(sPT2l + pp * 8);
#pragma unroll
                    for (int i2 = 0; i2 < 4; ++i2) {
                        const float4 ch = ch4[i2], cl = cl4[i2];  // points 2 i2, 2 i2 + 1 (duplicated)
                        p2 acc0 = {vh[2 * i2], vl[2 * i2]}, acc1 = {vh[2 * i2 + 1], vl[2 * i2 + 1]};
                        df_fma_acc2(acc0, Bp, {make_float2(ch.x, ch.y), make_float2(cl.x, cl.y)});
                        df_fma_acc2(acc1, Bp, {make_float2(ch.z, ch.w), make_float2(cl.z, cl.w)});
                        vh[2 * i2] = acc0.h;
                        vl[2 * i2] = acc0.l;
                        vh[2 * i2 + 1] = acc1.h;
                        vl[2 * i2 + 1] = acc1.l;
                    }
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const p2 nn = df_norm2({vh[i], vl[i]});
                    vh[i] = nn.h;
                    vl[i] = nn.l;
                }
            } else {
                for (uint32_t tk = 0; tk < n_e; ++tk) {
                    const int2 kv = skl[tk];
                    const int m = kv.x, pp = m & 7, qq = (m >> 3) & 7, rr = m >> 6;
                    const float cs = __int_as_float(kv.y) * qu;  // c 2^s, exact
                    const float fj = cs * sPTh[qq * 8 + j];
                    const float2 b = make_float2(fj * sPTh[rr * 8 + k0], fj * sPTh[rr * 8 + k0 + 4]);
                    const float4* ch4 = reinterpret_cast<const float4*>(sPT2h + pp * 8);
#pragma unroll
                    for (int i2 = 0; i2 < 4; ++i2) {
                        const float4 ch = ch4[i2];
                        vh[2 * i2] = f2fma(b, make_float2(ch.x, ch.y), vh[2 * i2]);
                        vh[2 * i2 + 1] = f2fma(b, make_float2(ch.z, ch.w), vh[2 * i2 + 1]);
                    }
                }
            }
        } else if constexpr (DF) {
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int r = 0; r < 8; ++r)
                    tb[(lane + 32 * s) * 9 + r] =
                        ((smask[s + 2 * r] >> lane) & 1u) ? (((s ? a2[r].y : a2[r].x) * qd + 12582912.0f) - 12582912.0f) * qu : 0.0f;
            dense_inverse_pairs(tb2, A.tab.Ph, A.tab.Pl);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float2 v0 = tb2[lane * 9 + i], v1 = tb2[(lane + 32) * 9 + i];
                const p2 d = df_sub2({vh[i], vl[i]}, {make_float2(v0.x, v1.x), make_float2(v0.y, v1.y)});
                vh[i] = d.h;
                vl[i] = d.l;
            }
            __syncwarp();
        } else {
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int r = 0; r < 8; ++r)
                    tb[(lane + 32 * s) * 9 + r] =
                        ((smask[s + 2 * r] >> lane) & 1u) ? (((s ? a2[r].y : a2[r].x) * qd + 12582912.0f) - 12582912.0f) * qu : 0.0f;
            dense_inverse_f32(tb, A.tab.Ph);
#pragma unroll
            for (int i = 0; i < 8; ++i) vh[i] = make_float2(tb[lane * 9 + i], tb[(lane + 32) * 9 + i]);
            __syncwarp();
        }

        // ---- errors of the lane's points: e2 = sum w d^2, Linf = max |d|, d = u - u~
        f2 e2;
        float lh = 0.0f, ll = 0.0f;  // Linf as a pair (|dh| first, then the signed low word)
        if constexpr (DF) {
            p2 ep = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const p2 d = {vh[i], vl[i]};
                const float4 w = sWq4[i * 32 + lane];
                const float2 ph = f2mul(d.h, d.h);
                const float2 pl = f2fma(d.h, f2add(d.l, d.l), f2fma(d.h, d.h, f2neg(ph)));
                df_fma_acc2(ep, {make_float2(w.x, w.y), make_float2(w.z, w.w)}, {ph, pl});
                lh = fmaxf(lh, fmaxf(fabsf(d.h.x), fabsf(d.h.y)));
            }
            ep = df_norm2(ep);
            e2 = warp_sum_pair(df_add({ep.h.x, ep.l.x}, {ep.h.y, ep.l.y}));
            const float LH = warp_max_nonneg(lh);
            // Linf = max |d| over normalised pairs, ordered by (|dh|, low word signed like dh):
            // only points whose |dh| is the element's largest can hold it
            ll = -FLT_MAX;
            if (lh == LH) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const p2 d = {vh[i], vl[i]};
                    if (fabsf(d.h.x) == LH)
                        ll = fmaxf(ll, __uint_as_float(__float_as_uint(d.l.x) ^ (__float_as_uint(d.h.x) & 0x80000000u)));
                    if (fabsf(d.h.y) == LH)
                        ll = fmaxf(ll, __uint_as_float(__float_as_uint(d.l.y) ^ (__float_as_uint(d.h.y) & 0x80000000u)));
                }
            }
            // largest low word among the lanes holding LH: order-preserving integer key of a float
            const uint32_t kb_ = (lh == LH) ? (__float_as_uint(ll) ^ ((__float_as_uint(ll) >> 31) ? 0xffffffffu : 0x80000000u)) : 0u;
            const uint32_t kmax = __reduce_max_sync(FULL, kb_);
            lh = LH;
            ll = __uint_as_float((kmax >> 31) ? (kmax ^ 0x80000000u) : ~kmax);
            if (LH == 0.0f) ll = 0.0f;
        } else {
            float2 ep = make_float2(0.0f, 0.0f);
            float dm = 0.0f;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float2 d = f2sub(uh[i], vh[i]);
                ep = f2fma(f2mul(A.tab.w2[i], d), d, ep);
                dm = fmaxf(dm, fmaxf(fabsf(d.x), fabsf(d.y)));
            }
            e2 = {warp_sum_f(fmaf(ep.x, wjk.x, ep.y * wjk.y)), 0.0f};
            lh = warp_max_nonneg(dm);
        }
        if (p.write_recon && p.recon[f] && eok) {  // FP64 mode: u~ = u - d' 2^ke, u reread from global
            const double sc = pow2d(s_res[il].ke);     // memory; the FP32 form: u~ = u~' 2^ke (exact)
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const uint64_t o = static_cast<uint64_t>(e) * WN3 + (lane + 32 * s) * 8;
                double2* dst = reinterpret_cast<double2*>(p.recon[f] + o);
#pragma unroll
                for (int i = 0; i < 8; i += 2) {
                    const float h0 = s ? vh[i].y : vh[i].x, l0 = s ? vl[i].y : vl[i].x;
                    const float h1 = s ? vh[i + 1].y : vh[i + 1].x, l1 = s ? vl[i + 1].y : vl[i + 1].x;
                    const double2 v = make_double2((static_cast<double>(h0) + static_cast<double>(l0)) * sc,
                                                   (static_cast<double>(h1) + static_cast<double>(l1)) * sc);
                    if constexpr (DF) {
                        const double2 u = reinterpret_cast<const double2*>(p.fields[f] + o)[i / 2];
                        dst[i / 2] = make_double2(u.x - v.x, u.y - v.y);
                    } else {
                        dst[i / 2] = v;
                    }
                }
            }
        }

        if (lane == 0) {
            WStash& st = s_res[il];
            const bool zero = st.hmax < 0x00100000u;  // zeros and subnormals only: a zero block
            st.sh = zero ? 0.0f : S.h;
            st.sl = zero ? 0.0f : S.l;
            st.eh = zero ? 0.0f : e2.h;
            st.el = zero ? 0.0f : e2.l;
            st.lh = zero ? 0.0f : lh;
            st.ll = zero ? 0.0f : ll;
        }
        __syncwarp();  // the kept list and mask words are reused by the next element
    }
    if (threadIdx.x == 0) {
        s_tile[1] = atomicAdd(counter, 1u);
        resolve(s_tile[1], 1);
    }
    __syncthreads();  // every element of the tile is done
    {  // this warp's first block of the next tile streams in during the tile's bookkeeping
        if (s_tile[1] < total_tiles && !s_abort) {
            const uint32_t itn = s_titem[1], tn = s_tloc[1];
            const LaunchParams* pn = BATCH ? &q.items[itn] : &A.p;
            uint32_t fn, e0n;
            int nhn;
            geom(tn, static_cast<uint32_t>(pn->tiles_per_field), static_cast<uint32_t>(pn->n_elem), fn, e0n, nhn);
            if (wid < nhn) {
                if (lane == 0) {
                    fence_proxy_async();
                    issue(BATCH ? &qmaps[q.field_base[itn] + fn] : &A.tm[fn], e0n + static_cast<uint32_t>(wid));
                }
                inflight = true;
            }
        }
    }
    constexpr int EPL = kWarpTile / 32;  // tile bookkeeping: elements per lane
    static_assert(kWarpTile % 32 == 0, "tile of whole warps");
    if (wid == 0) {
        // tile aggregate and within-tile prefixes (lane l: elements EPL l .. EPL l + EPL - 1),
        // published now; the look-back runs one tile later (for tile t_prev here), when the tiles
        // before it have almost always finished, so it rarely waits
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
            pre[EPL * lane + h] = run;
            run += cl[h];
        }
        const uint32_t tot = __shfl_sync(FULL, incl, 31);
        if (lane == 0 && bchk(tcur < static_cast<uint32_t>(p.n_fields) * tpf, status)) {
            pre[kWarpTile] = tot;
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
    {
        // every warp: FP64 partials and element report of its own elements (lane k: element
        // wid + 4k), so the FP64 conversions run on all four SMSPs' FP64 units at once
        static_assert(kWarpTile == 32 * WPB, "one element of the tile per lane of each warp");
        double v0 = 0.0, v1 = 0.0;
        unsigned long long m2 = 0ull, m3 = 0ull;  // maxima of non-negative doubles as bit patterns
        const int il = wid + WPB * lane;
        if (il < nh) {
            const WStash st = s_res[il];
            const uint64_t ge = static_cast<uint64_t>(f) * E + e0 + il;
            const double J = p.jac[e0 + il];
            // back from the prescaled block: energies times 2^2ke (two exact factors), Linf times 2^ke
            const double sc = pow2d(st.ke);
            const double Sd = ((static_cast<double>(st.sh) + static_cast<double>(st.sl)) * sc) * sc;
            const double e2d = ((static_cast<double>(st.eh) + static_cast<double>(st.el)) * sc) * sc;
            v0 = J * e2d;
            v1 = J * Sd;
            const double x2 = (static_cast<double>(st.lh) + static_cast<double>(st.ll)) * sc;
            m2 = static_cast<unsigned long long>(__double_as_longlong(x2));
            m3 = st.hmax;
            const bool gok = bchk(ge < static_cast<uint64_t>(p.n_fields) * E, status);
            if (gok) p.hmax_elem[ge] = st.hmax;
            if (p.elem_report && gok) {
                double* er = p.elem_report + 3 * ge;
                er[0] = v0;
                er[1] = v1;
                er[2] = x2;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v0 += __shfl_down_sync(FULL, v0, o);
            v1 += __shfl_down_sync(FULL, v1, o);
            m2 = max(m2, __shfl_down_sync(FULL, m2, o));
            m3 = max(m3, __shfl_down_sync(FULL, m3, o));
        }
        if (lane == 0) {
            s_wpart[wid][0] = v0;
            s_wpart[wid][1] = v1;
            s_wpart[wid][2] = __longlong_as_double(static_cast<long long>(m2));
            s_wpart[wid][3] = static_cast<double>(m3);  // the largest high word, as a number
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && bchk(tcur < static_cast<uint32_t>(p.n_fields) * tpf, status)) {
        // tile partials: the warps' partials in a fixed order
        double* tp = p.tile_part + 4ull * tcur;
        tp[0] = ((s_wpart[0][0] + s_wpart[1][0]) + s_wpart[2][0]) + s_wpart[3][0];
        tp[1] = ((s_wpart[0][1] + s_wpart[1][1]) + s_wpart[2][1]) + s_wpart[3][1];
        tp[2] = fmax(fmax(s_wpart[0][2], s_wpart[1][2]), fmax(s_wpart[2][2], s_wpart[3][2]));
        tp[3] = fmax(fmax(s_wpart[0][3], s_wpart[1][3]), fmax(s_wpart[2][3], s_wpart[3][3]));
    }
    if (t_prev != 0xffffffffu) place_codes(pprev, par ^ 1, nh_prev, s_excl);  // the previous tile's codes
    if (recomputed && lane == 0) atomicAdd(&p.ctl->recomputed, recomputed);
    recomputed = 0;
    t_prev = tcur;
    nh_prev = nh;
    par ^= 1;
    if (s_abort) break;
    tag = (tag + 1 == 0xffffu) ? 0u : tag + 1;
    __syncwarp();
    }
    // the last tile: its look-back, then its codes
    if (t_prev != 0xffffffffu && !s_abort) {
        const LaunchParams& pl = BATCH ? s_par[par ^ 1] : A.p;
        if (wid == 0) {
            const uint64_t excl = lookback_warp(pl.tile_state, t_prev, tot_prev, &pl.ctl->status);
            if (lane == 0) s_excl = excl;
        }
        __syncthreads();
        place_codes(pl, par ^ 1, nh_prev, s_excl);
    }
    // after an abort: let a requested block land before the CTA exits
    if (inflight && !mbar_wait_bounded(bar, parity)) drain_stage(bar, parity, &(BATCH ? s_par[par ^ 1] : A.p).ctl->status);
    // a single launch finalizes in the CTA that finishes last (no separate kernel, which could wait
    // behind another launch's persistent CTAs), one field per warp
    if constexpr (!BATCH) {
        if (last_cta_done(&A.p.ctl->done_ctas))
            for (int f = wid; f < A.p.n_fields; f += WPB) finalize_field_warp(A.p, f, WLX, kWarpTile);
    }
}

// One warp per (item, field) of a batched launch, eight per block: the fixed-order finalize of a
// single launch's last CTA, so a batched snapshot's reports equal its single launch's bit for bit.
__global__ void __launch_bounds__(256) finalize_warp_batch_kernel(const BatchQueue q, uint32_t total_fields) {
    const uint32_t gf = blockIdx.x * 8u + (threadIdx.x >> 5);
    if (gf >= total_fields) return;  // uniform over the warp
    int lo = 0, hi = q.n_items - 1;  // last item with field_base <= gf
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (q.field_base[mid] <= gf) lo = mid; else hi = mid - 1;
    }
    finalize_field_warp(q.items[lo], static_cast<int>(gf - q.field_base[lo]), WLX, kWarpTile);
}

// ------------------------------------------------------------ host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
    });
    return fn;
}

WTables make_wtables() {
    WTables t;
    double Am[64], Phi[64], w[8];
    basis_tables(8, Am, Phi, w);
    for (int i = 0; i < 64; ++i) {
        t.A2[i] = make_float2(static_cast<float>(Am[i]), static_cast<float>(Am[i]));
        t.A64[i] = Am[i];
        t.Ah[i] = static_cast<float>(Am[i]);
        t.Al[i] = static_cast<float>(Am[i] - static_cast<double>(t.Ah[i]));
        t.Ph[i] = static_cast<float>(Phi[i]);
        t.Pl[i] = static_cast<float>(Phi[i] - static_cast<double>(t.Ph[i]));
    }
    for (int i = 0; i < 8; ++i) {
        t.wh[i] = static_cast<float>(w[i]);
        t.wl[i] = static_cast<float>(w[i] - static_cast<double>(t.wh[i]));
        t.w2[i] = make_float2(t.wh[i], t.wh[i]);
    }
    return t;
}

template <int MODE, bool BATCH, bool CUM = false>
int launch_mode(const WArgs& a, const BatchQueue& q, uint64_t total_tiles, uint64_t stage_ctas, void* stream) {
    using SM = WSmem<MODE != 0>;
    cudaError_t err;
    auto kern = reduce_warp_kernel<MODE, BATCH, CUM>;
    if ((err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes)) != cudaSuccess)
        return (int)err;
    int dev = 0, sms = 0, per_sm = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return (int)err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WPB * 32, SM::bytes)) != cudaSuccess)
        return (int)err;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    // persistent: as many CTAs as fit at once, never more than tiles or staging slots
    const uint64_t want = std::min<uint64_t>(total_tiles, stage_ctas);
    const unsigned grid = (unsigned)std::min<uint64_t>(want, static_cast<uint64_t>(sms) * per_sm);
    if (grid == 0) return (int)cudaErrorInvalidConfiguration;
    kern<<<grid, WPB * 32, SM::bytes, static_cast<cudaStream_t>(stream)>>>(a, q);
    return (int)cudaGetLastError();
}

// Self-test of the bounded waits: the look-back of tile 1, whose predecessor never
// publishes, and phase 0 of an mbarrier that expects one arrival that never comes.
// Each wait gives up at its bound and records SEMR_STATUS_TIMEOUT; nothing faults or hangs.
__global__ void selftest_waits_kernel(uint64_t* tile_state, unsigned* status) {
    __shared__ uint64_t bar;
    const int lane = threadIdx.x & 31;
    lookback_warp(tile_state, 1, 0, &status[0]);
    if (lane == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (!mbar_wait_bounded(&bar, 0)) {  // as the reduce kernel's abort path: timeout, then the drain
        if (lane == 0) atomicOr(&status[1], static_cast<unsigned>(SEMR_STATUS_TIMEOUT));
        drain_stage(&bar, 0, &status[1]);
    }
}

}  // namespace

bool warp_applicable(const LaunchParams& p) {
    if (p.lx != 8 || p.lossless || p.width != 2) return false;
    if (p.precision != SEMR_FP64 && p.precision != SEMR_FP32) return false;
    if (static_cast<uint64_t>(p.n_elem) * WNP >= (1ull << 31)) return false;  // TMA row coordinate
    for (int f = 0; f < p.n_fields; ++f)
        if (reinterpret_cast<uintptr_t>(p.fields[f]) & 15u) return false;  // TMA needs 16-byte aligned blocks
    return encoder() != nullptr;
}

int launch_reduce_warp(const LaunchParams& p, void* stream) {
    EncodeTiledFn enc = encoder();
    if (!enc) return (int)cudaErrorNotSupported;
    WArgs a;
    std::memset(&a, 0, sizeof(a));
    a.p = p;
    a.tab = make_wtables();
    a.tau_h = static_cast<float>(p.tau);
    a.tau_l = static_cast<float>(p.tau - static_cast<double>(a.tau_h));
    a.n_elem = static_cast<uint32_t>(p.n_elem);
    a.tiles_per_field = static_cast<uint32_t>(p.tiles_per_field);
    a.total_tiles = static_cast<uint32_t>(static_cast<uint64_t>(p.n_fields) * p.tiles_per_field);
    for (int f = 0; f < p.n_fields; ++f) {
        const cuuint64_t dims[2] = {8, static_cast<cuuint64_t>(p.n_elem) * WNP};
        const cuuint64_t strides[1] = {64};
        const cuuint32_t box[2] = {8, WNP};
        const cuuint32_t estr[2] = {1, 1};
        if (enc(&a.tm[f], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(p.fields[f]), dims, strides, box,
                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return (int)cudaErrorInvalidValue;
    }
    BatchQueue q{};
    if (p.cumulative)  // cumulative-energy truncation (single launches only)
        return p.precision == SEMR_FP32 ? launch_mode<0, false, true>(a, q, a.total_tiles, p.stage_ctas, stream)
                                        : launch_mode<1, false, true>(a, q, a.total_tiles, p.stage_ctas, stream);
    return p.precision == SEMR_FP32 ? launch_mode<0, false>(a, q, a.total_tiles, p.stage_ctas, stream)
                                    : launch_mode<1, false>(a, q, a.total_tiles, p.stage_ctas, stream);
}

int warp_encode_maps(const LaunchParams& p, void* maps) {
    EncodeTiledFn enc = encoder();
    if (!enc) return (int)cudaErrorNotSupported;
    for (int f = 0; f < p.n_fields; ++f) {
        const cuuint64_t dims[2] = {8, static_cast<cuuint64_t>(p.n_elem) * WNP};
        const cuuint64_t strides[1] = {64};
        const cuuint32_t box[2] = {8, WNP};
        const cuuint32_t estr[2] = {1, 1};
        CUtensorMap* tm = reinterpret_cast<CUtensorMap*>(static_cast<uint8_t*>(maps) + kTensorMapBytes * f);
        if (enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(p.fields[f]), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return (int)cudaErrorInvalidValue;
    }
    return 0;
}

int launch_reduce_warp_batch(const BatchQueue& q, int precision, bool cumulative, uint64_t stage_ctas, void* stream) {
    WArgs a;
    std::memset(&a, 0, sizeof(a));
    a.tab = make_wtables();
    if (cumulative)
        return precision == SEMR_FP32 ? launch_mode<0, true, true>(a, q, q.total_tiles, stage_ctas, stream)
                                      : launch_mode<1, true, true>(a, q, q.total_tiles, stage_ctas, stream);
    return precision == SEMR_FP32 ? launch_mode<0, true>(a, q, q.total_tiles, stage_ctas, stream)
                                  : launch_mode<1, true>(a, q, q.total_tiles, stage_ctas, stream);
}

int launch_finalize_warp_batch(const BatchQueue& q, uint32_t total_fields, void* stream) {
    finalize_warp_batch_kernel<<<(total_fields + 7) / 8, 256, 0, static_cast<cudaStream_t>(stream)>>>(q, total_fields);
    return (int)cudaGetLastError();
}


}  // namespace semr

extern "C" int semr_selftest_waits(uint32_t* status_out) {
    if (!status_out) return SEMR_EINVAL;
    void* buf = nullptr;
    if (cudaMalloc(&buf, 32) != cudaSuccess) return SEMR_ENOMEM;
    int rc = SEMR_OK;
    uint64_t* tile_state = static_cast<uint64_t*>(buf);            // 2 states, never published
    unsigned* status = reinterpret_cast<unsigned*>(tile_state + 2);  // 2 status words
    if (cudaMemset(buf, 0, 32) != cudaSuccess) rc = SEMR_ECUDA;
    if (rc == SEMR_OK) {
        semr::selftest_waits_kernel<<<1, 32>>>(tile_state, status);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(status_out, status, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = SEMR_ECUDA;
    }
    cudaFree(buf);
    return rc;
}
