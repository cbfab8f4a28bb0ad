// Fast fused reduce kernel (arXiv 2407.20731, Sec. IV-B: JPEG-like spectral
// truncation of SEM fields; Eq. 1 for the compression ratio), built around
// B300's arithmetic: FP32 lanes run 65 TFLOP/s while every FP64 instruction
// (DFMA, DADD, F2F conversions, DMNMX) shares a pipe of under 1 TFLOP/s.  So
// no FP64 instruction runs per point:
//   * MODE_F32  (the precision form): FP32 transforms with FP32 accumulation.
//   * MODE_DF64 (FP64 accuracy): the forward transform in FP32 under a proven
//     error bound, every coefficient whose keep or rounding decision that bound
//     cannot settle recomputed in hardware FP64 (rare), and the energy,
//     reconstruction and norms as pairs of floats (hi + lo, about 48
//     significant bits, error-free products via FMA), which agree with FP64 to
//     ~1e-14 relative.
// The input doubles are split into floats with integer instructions, each
// element read as u 2^-ke (an exact power-of-two prescale).  The
// threshold test is an exact magnitude comparison, the sums over an element
// are pair-of-float tree sums (deterministic), and only once per element do
// a few FP64 instructions form t = tau S_e, the step and the threshold.
//
// Cumulative-energy truncation (MODE_CUM): the modes kept are those whose
// energy is at least T, the smallest energy value v with
//   sum of all energies <= v  >  t = tau S_e,
// which is exactly what sorting the energies and dropping the longest
// prefix whose sum fits the budget t selects (equal energies kept together),
// without a sort.  Energies become 64-bit fixed-point keys floor(a^2 2^K),
// t 2^K in [2^47, 2^48), so every sum is an exact integer sum (deterministic
// in any order): an octave histogram of key sums (shared atomics) finds the
// octave that holds T, one warp sorts that octave's few keys (or bisects
// when there are more than 32) and scans them against the budget.  FP64
// mode computes the forward transform in float pairs for this variant: the
// boundary depends on the sum of every small energy, which FP32 coefficients
// cannot settle.
//
// The reconstruction exploits how few modes survive (2-3 per element at
// tau = 1e-3): each thread rebuilds its pencil from the element's list of
// kept modes, u~(i) = sum_m c_m 2^s phi_p(x_i) phi_q(x_j) phi_r(x_k).  When a
// tile keeps many modes (or in lossless mode) it switches to the dense
// folded inverse with two shared-memory transposes.
#include <algorithm>
#include <type_traits>

#include "semr_device.cuh"

namespace semr {

constexpr int MODE_F32 = 0;
constexpr int MODE_DF64 = 1;  // bit 0: float-pair (FP64-accurate) arithmetic
constexpr int MODE_CUM = 2;   // bit 1: cumulative-energy truncation

template <int LX>
struct FastTables {
    float Ah[LX * LX], Al[LX * LX];    // analysis A[p*LX + i] (hi, lo)
    double A64[LX * LX];               // analysis A[p*LX + i] in FP64 (the exact recomputation)
    float Ph[LX * LX], Pl[LX * LX];    // synthesis Phi[i*LX + p] (hi, lo)
    float wh[LX], wl[LX];              // GLL weights (hi, lo)
};

template <int LX, int TILE_>
struct FCfg {
    static constexpr int NP = LX * LX;             // threads (pencils) per element
    static constexpr int N3 = LX * LX * LX;
    static constexpr int TILE = TILE_;             // elements per tile
    static constexpr int NT = TILE * NP;
    static constexpr int BLOCK = (NT + 31) / 32 * 32;
    static constexpr int NW = BLOCK / 32;
    static constexpr int MW = (N3 + 31) / 32;      // 32-bit mask words per element
    static constexpr int SY = LX + 1;              // padded transpose strides
    static constexpr int SX = LX * (LX + 1);
    static constexpr int BUFN = LX * SX;
    static constexpr int PT = LX + 1;              // padded row of the shared Phi tables
    // Elements line up with warps: whole warps (NP % 32 == 0) or a power-of-two
    // lane group inside one warp (32 % NP == 0).  Then reductions run on warp
    // shuffles and the mask is built with ballots; otherwise through shared memory.
    static constexpr bool ALIGNED = (NP % 32 == 0) || (32 % NP == 0);
    static constexpr int SEG = NP < 32 ? NP : 32;  // lanes of one element in a warp
    static constexpr int WPE = NP >= 32 ? NP / 32 : 1;
    static constexpr bool BALLOT = (NP % 32 == 0);
};

// Coefficients per tile whose decisions are recomputed exactly in one round.
constexpr int AMB_CAP = 64;

// Sparse reconstruction from the kept-mode list while no element of the tile
// keeps more modes than this; the dense folded inverse otherwise.
__host__ __device__ constexpr int sparse_max(int mode) { return (mode & 1) ? 12 : 5; }

template <int LX, int MODE, int TILE_>
struct FSmem {
    using C = FCfg<LX, TILE_>;
    static constexpr size_t vb = (MODE & MODE_DF64) ? 8 : 4;   // float2 or float per value
    static constexpr size_t buf_bytes = vb * C::TILE * C::BUFN;
    static constexpr size_t off_t1 = 0;
    static constexpr size_t off_t2 = off_t1 + buf_bytes;
    // code staging: 8 B per code for lossless FP32 codes and the cumulative keys,
    // 4 B in FP64 threshold mode (its lossless form runs on the hardware-FP64 kernel)
    static constexpr size_t code_b = (MODE == 1) ? 4 : 8;
    static constexpr int KL = sparse_max(MODE) < C::N3 ? sparse_max(MODE) : C::N3;  // kept-list entries per element
    static constexpr size_t off_codes = off_t2 + buf_bytes;
    static constexpr size_t off_kc = off_codes + code_b * C::TILE * C::N3;  // kept codes (f32)
    static constexpr size_t off_km = off_kc + 4ull * C::TILE * KL;          // kept modes (u16)
    // reduction slots: one per (warp, element segment) when elements line up with warps, else one per thread
    static constexpr int RED_N = C::ALIGNED ? C::NW * (32 / C::SEG) : C::BLOCK;
    static constexpr size_t off_red = (off_km + 2ull * C::TILE * KL + 15) / 16 * 16;  // RED_N x 16 B
    static constexpr size_t off_elem = off_red + 16ull * RED_N;            // TILE x 8 doubles
    static constexpr size_t off_phi = off_elem + 64ull * C::TILE;          // 4 tables x LX x PT floats
    static constexpr size_t off_amat = off_phi + 16ull * LX * C::PT;       // 2 tables x LX x PT floats
    static constexpr size_t off_amb = off_amat + 8ull * LX * C::PT;        // AMB_CAP entries + values
    static constexpr size_t off_wq = (off_amb + 12ull * AMB_CAP + 4ull * C::TILE + 16 + 15) / 16 * 16;
    static constexpr size_t off_mask = off_wq + ((MODE & MODE_DF64) ? 8ull * C::NP * LX : 0);  // TILE x MW u32
    static constexpr size_t off_wpre = off_mask + 4ull * C::TILE * C::MW;
    static constexpr size_t off_misc = (off_wpre + 4ull * C::TILE * C::MW + 15) / 16 * 16;
    // cumulative variant: per element 64 octave sums (unless one warp holds all
    // the keys), then boundary key, base sum, budget, octave, count, K
    static constexpr bool CUM_DIRECT = C::N3 <= 32;
    static constexpr size_t off_cum = (off_misc + 4ull * (9 * C::TILE + 16) + 15) / 16 * 16;
    static constexpr size_t cum_bytes = (MODE & MODE_CUM) ? (CUM_DIRECT ? 0 : 512ull * C::TILE) + 40ull * C::TILE : 0;
    static constexpr size_t bytes = off_cum + cum_bytes;
};

// Per-element reduction of one sum (a float pair) and one maximum (a 64-bit
// pattern of a non-negative number, read back as a double or as a float).
// Results: out[lt*8 + slot_sum], out[lt*8 + slot_max] (doubles).  The sum is
// a pair-of-float tree in FP64 mode, an FP32 tree inside a warp in FP32 mode;
// partials across warps are added in FP64.  Fixed order: deterministic.
template <int LX, int TILE_, bool DF>
__device__ __forceinline__ void elem_reduce(float* red, double* out, f2 s, unsigned long long mx, bool mx_double,
                                            int slot_sum, int slot_max, int n_here) {
    using C = FCfg<LX, TILE_>;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if constexpr (C::ALIGNED) {
#pragma unroll
        for (int o = C::SEG / 2; o > 0; o >>= 1) {
            const float h = __shfl_xor_sync(0xffffffffu, s.h, o);
            if constexpr (DF) {
                const float l = __shfl_xor_sync(0xffffffffu, s.l, o);
                const f2 t = two_sum(s.h, h);
                s = {t.h, t.l + (s.l + l)};
            } else {
                s.h += h;
            }
        }
        const unsigned seg_mask = (C::SEG == 32) ? 0xffffffffu : (((1u << C::SEG) - 1u) << (lane & ~(C::SEG - 1)));
        unsigned mhi = (unsigned)(mx >> 32), mlo = (unsigned)mx;
        if (mx_double) {
            const unsigned top = __reduce_max_sync(seg_mask, mhi);
            mlo = __reduce_max_sync(seg_mask, mhi == top ? mlo : 0u);
            mhi = top;
        } else {
            mlo = __reduce_max_sync(seg_mask, mlo);
            mhi = 0;
        }
        float4* r4 = reinterpret_cast<float4*>(red);
        const int slot = warp * (32 / C::SEG) + lane / C::SEG;  // one slot per (warp, element segment)
        if ((lane & (C::SEG - 1)) == 0) r4[slot] = make_float4(s.h, s.l, __uint_as_float(mhi), __uint_as_float(mlo));
        __syncthreads();
        if (tid < C::TILE && tid < n_here) {
            double sum = 0.0;
            unsigned long long m = 0;
            for (int k = 0; k < C::WPE; ++k) {
                const float4 v = r4[tid * C::WPE + k];
                sum += (double)v.x + (double)v.y;
                m = max(m, ((unsigned long long)__float_as_uint(v.z) << 32) | __float_as_uint(v.w));
            }
            out[tid * 8 + slot_sum] = sum;
            out[tid * 8 + slot_max] = mx_double ? __longlong_as_double((long long)m) : (double)__uint_as_float((unsigned)m);
        }
        __syncthreads();
    } else {
        float4* r4 = reinterpret_cast<float4*>(red);
        r4[tid] = make_float4(s.h, s.l, __uint_as_float((unsigned)(mx >> 32)), __uint_as_float((unsigned)mx));
        __syncthreads();
        for (int lt = warp; lt < C::TILE; lt += C::NW) {
            f2 a = {0.0f, 0.0f};
            unsigned long long m = 0;
            for (int i = lane; i < C::NP; i += 32) {
                const float4 v = r4[lt * C::NP + i];
                a = df_add(a, {v.x, v.y});
                m = max(m, ((unsigned long long)__float_as_uint(v.z) << 32) | __float_as_uint(v.w));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a = df_add(a, {__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)});
                m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
            }
            if (lane == 0) {
                out[lt * 8 + slot_sum] = (double)a.h + (double)a.l;
                out[lt * 8 + slot_max] =
                    mx_double ? __longlong_as_double((long long)m) : (double)__uint_as_float((unsigned)m);
            }
        }
        __syncthreads();
    }
}

// Resident threads per SM the register budget aims at: enough warps to hide
// the latency of the tile's barrier phases, without spilling the larger orders.
// FP64 mode with 2-element tiles (lx >= 9), measured: 768 threads (3 CTAs at lx
// 9-10, 2 at lx 12) beat 512; at lx = 11 the third CTA's register cap spills.
// The cumulative variant: 1024 threads in the FP32 form; in FP64 mode 1024 up to
// lx = 6 and 768 above (measured at lx = 6, 8 and 10 against 512 and 768).
constexpr int min_ctas_per_sm(int lx, int mode, int block) {
    const int target = (mode & MODE_CUM) ? (!(mode & MODE_DF64) ? 1024 : (lx <= 6 ? 1024 : 768))
                       : !(mode & MODE_DF64) ? (lx <= 10 ? 1024 : 768)
                                             : (lx <= 8 ? 1024 : lx == 11 ? 512 : 768);
    return target / block > 0 ? target / block : 1;
}

// BATCH = false: one reduction, parameters p0.  BATCH = true: the work queue
// q of several reductions of this lx (each with its own payload and scratch).
template <int LX, int MODE, int TILE_, bool BATCH>
__global__ void __launch_bounds__(FCfg<LX, TILE_>::BLOCK, min_ctas_per_sm(LX, MODE, FCfg<LX, TILE_>::BLOCK))
reduce_fast_kernel(const LaunchParams p0, const BatchQueue q, const FastTables<LX> tab) {
    using C = FCfg<LX, TILE_>;
    using S = FSmem<LX, MODE, TILE_>;
    constexpr int NP = C::NP, N3 = C::N3, TILE = C::TILE, MW = C::MW, SX = C::SX, SY = C::SY, PT = C::PT;
    constexpr int CS = (LX % 4 == 0) ? LX : PT;  // row stride of the column table (16-byte rows when possible)
    constexpr bool DF = (MODE & MODE_DF64) != 0;
    constexpr bool CUM = (MODE & MODE_CUM) != 0;
    constexpr bool DIRECT = S::CUM_DIRECT;  // cumulative: one warp holds all keys of an element
    using V = typename std::conditional<DF, float2, float>::type;  // one transposed value
    // dense inverse once any element of the tile keeps more modes than this
    constexpr int SPARSE_MAX = sparse_max(MODE);
    constexpr int KL = S::KL;

    extern __shared__ __align__(16) uint8_t smem[];
    V* t1 = reinterpret_cast<V*>(smem + S::off_t1);
    V* t2 = reinterpret_cast<V*>(smem + S::off_t2);
    uint8_t* scodes = smem + S::off_codes;
    float* skc = reinterpret_cast<float*>(smem + S::off_kc);
    uint16_t* skm = reinterpret_cast<uint16_t*>(smem + S::off_km);
    float* red = reinterpret_cast<float*>(smem + S::off_red);
    double* selem = reinterpret_cast<double*>(smem + S::off_elem);
    float* sPh = reinterpret_cast<float*>(smem + S::off_phi);  // Phi[i][p], rows padded
    float* sPl = sPh + LX * PT;
    float* sPTh = sPl + LX * PT;                                 // Phi[i][p] stored as [p][i]
    float* sPTl = sPTh + LX * PT;
    float* sAh = reinterpret_cast<float*>(smem + S::off_amat);  // A[p][i], rows padded
    float* sAl = sAh + LX * PT;
    int* s_amb = reinterpret_cast<int*>(smem + S::off_amb);          // [AMB_CAP]: (element << 16) | mode
    float* s_ambv = reinterpret_cast<float*>(s_amb + AMB_CAP);       // [2 * AMB_CAP]: exact values
    int* s_namb = reinterpret_cast<int*>(s_ambv + 2 * AMB_CAP);      // [1 + TILE]: count, per-element flags
    float2* sWq = reinterpret_cast<float2*>(smem + S::off_wq);        // [LX][NP] weight products (pairs)
    float* t1f = reinterpret_cast<float*>(smem + S::off_t1);         // FP32 views of the transpose buffers
    float* t2f = reinterpret_cast<float*>(smem + S::off_t2);
    uint32_t* smask = reinterpret_cast<uint32_t*>(smem + S::off_mask);
    uint32_t* swpre = reinterpret_cast<uint32_t*>(smem + S::off_wpre);
    int* smisc = reinterpret_cast<int*>(smem + S::off_misc);
    unsigned long long* s_tile = reinterpret_cast<unsigned long long*>(smisc);  // [0] tile, [1] excl
    int* s_cnt = smisc + 4;              // [TILE]
    int* s_epre = s_cnt + TILE;          // [TILE + 1]
    int* s_step = s_epre + TILE + 1;     // [TILE]
    int* s_mode = s_step + TILE;         // [TILE]
    uint32_t* s_hx = reinterpret_cast<uint32_t*>(s_mode + TILE);  // [TILE] largest high word of |u|
    int* s_flag = reinterpret_cast<int*>(s_hx + TILE);  // [2]: dense inverse needed
    float* s_g = reinterpret_cast<float*>(s_flag + 2);  // [2 * TILE]: threshold (hi, lo)
    float* s_marg = s_g + 2 * TILE;                       // [TILE]: bound on |a_fp32 - a|
    // cumulative variant
    unsigned long long* sbk = reinterpret_cast<unsigned long long*>(smem + S::off_cum);  // [TILE][64] octave sums
    unsigned long long* s_T = sbk + (DIRECT ? 0 : 64 * TILE);  // [TILE] smallest kept key (~0: none)
    unsigned long long* s_base = s_T + TILE;                    // [TILE] key sum below the octave of T
    unsigned long long* s_tint = s_base + TILE;                 // [TILE] floor(t 2^K)
    int* s_bstar = reinterpret_cast<int*>(s_tint + TILE);       // [TILE] octave (bit length) of T
    int* s_ncand = s_bstar + TILE;                              // [TILE] keys in that octave
    int* s_cK = s_ncand + TILE;                                 // [TILE] K
    unsigned long long* scand = reinterpret_cast<unsigned long long*>(scodes);  // [TILE][N3] keys of the octave

    // parameters of the reduction the current tile belongs to
    __shared__ LaunchParams sp;
    __shared__ int s_item;
    const LaunchParams& p = sp;
    constexpr int PW = sizeof(LaunchParams) / 4;
    static_assert(sizeof(LaunchParams) % 4 == 0, "descriptor copy by words");

    const int tid = threadIdx.x, lane = tid & 31;
    const int lt = tid / NP;
    const int P = tid % NP;
    const int pa = P / LX, pb = P % LX;
    const bool in_tile = lt < TILE;
    const int lts = in_tile ? lt : 0;
    V* b1 = t1 + lts * C::BUFN;
    V* b2 = t2 + lts * C::BUFN;

    for (int i = tid; i < LX * LX; i += C::BLOCK) {
        const int r = i / LX, c = i % LX;  // Phi[r][c]
        sPh[r * PT + c] = tab.Ph[i];
        sPl[r * PT + c] = tab.Pl[i];
        sPTh[c * CS + r] = tab.Ph[i];
        sPTl[c * CS + r] = tab.Pl[i];
        sAh[r * PT + c] = tab.Ah[i];
        sAl[r * PT + c] = tab.Al[i];
    }
    // quadrature weight products w_i w_j w_k of this pencil (j = pb, k = pa):
    // FP32 mode keeps them in registers, FP64 mode as pairs in a shared table
    float wq32[LX];
    {
        const f2 wjk = df_mul({tab.wh[pa], tab.wl[pa]}, {tab.wh[pb], tab.wl[pb]});
#pragma unroll
        for (int i = 0; i < LX; ++i) {
            if constexpr (DF) {
                const f2 w3 = df_mul({tab.wh[i], tab.wl[i]}, wjk);
                if (in_tile && lt == 0) sWq[i * NP + P] = make_float2(w3.h, w3.l);
                wq32[i] = 0.0f;
            } else {
                wq32[i] = tab.wh[i] * wjk.h;
            }
        }
    }

    if (!BATCH) {
        for (int i = tid; i < PW; i += C::BLOCK) reinterpret_cast<int*>(&sp)[i] = reinterpret_cast<const int*>(&p0)[i];
    }
    if (tid == 0) s_item = -1;
    const uint64_t total_tiles = BATCH ? q.total_tiles : (uint64_t)p0.n_fields * p0.tiles_per_field;
    unsigned* counter = BATCH ? q.counter : &p0.ctl->tile_counter;

    // persistent CTA: claim tiles in increasing order until none are left
    for (;;) {
    if (tid == 0) {
        const uint64_t g = atomicAdd(counter, 1u);
        uint64_t local = g;
        int item = 0;
        if (BATCH && g < total_tiles) {  // last item whose first tile is <= g
            int lo = 0, hi = q.n_items - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) / 2;
                if (q.tile_base[mid] <= g) lo = mid; else hi = mid - 1;
            }
            item = lo;
            local = g - q.tile_base[lo];
        }
        s_tile[0] = (g < total_tiles) ? local : ~0ull;
        s_flag[1] = item;
        s_flag[0] = 0;
    }
    if constexpr (!C::BALLOT) {
        for (int i = tid; i < TILE * MW; i += C::BLOCK) smask[i] = 0u;
    }
    if (tid < TILE) s_hx[tid] = 0u;
    __syncthreads();
    const uint64_t tile = s_tile[0];
    if (tile == ~0ull) break;
    if (BATCH && s_flag[1] != s_item) {  // load the item's parameters
        const int item = s_flag[1];
        __syncthreads();
        for (int i = tid; i < PW; i += C::BLOCK)
            reinterpret_cast<int*>(&sp)[i] = reinterpret_cast<const int*>(&q.items[item])[i];
        if (tid == 0) s_item = item;
        __syncthreads();
    }
    ScratchControl* ctl = p.ctl;
    uint64_t* tile_state = p.tile_state;
    double* tile_part = p.tile_part;
    const int width = p.width;
    const int f = (int)(tile / p.tiles_per_field);
    const int64_t e0 = (int64_t)(tile % p.tiles_per_field) * TILE;
    const int n_here = (p.n_elem - e0 < TILE) ? (int)(p.n_elem - e0) : TILE;
    const bool active = (tid < C::NT) && (lt < n_here);
    const int64_t e = e0 + lt;
    // bounds build: the tile, its elements and its field's section of the payload (every write
    // of the tile below is skipped if they fall outside their buffers)
    const bool tok = bchk(tile < (uint64_t)p.n_fields * p.tiles_per_field && f < p.n_fields && n_here >= 1 &&
                              pad16((uint64_t)p.n_elem * ((N3 + 7) / 8)) + 2 * pad16(2ull * p.n_elem) <= p.fixed_bytes &&
                              p.header_bytes + (f + 1ull) * p.fixed_bytes <= p.code_base &&
                              p.code_base <= p.payload_cap,
                          &p.ctl->status);

    // ---- load the pencil u[k=pa][j=pb][0..LX-1], split to floats with integer ops.  The
    // element is read as u 2^-ke, ke the binary exponent of its largest |u| (an exact
    // power-of-two prescale: masks and codes do not change under it, steps and norms are
    // scaled back exactly), so every value formed below lies near 1 whatever the field's units.
    float uh[LX], ul[LX];
    unsigned long long umax_bits = 0;  // max |u|: exact double pattern
    {
        double u[LX];
        if (active) {
            const double* src = p.fields[f] + e * N3 + P * LX;
            if constexpr ((LX % 2) == 0) {
#pragma unroll
                for (int i = 0; i < LX; i += 2) {
                    const double2 v = __ldg(reinterpret_cast<const double2*>(src + i));
                    u[i] = v.x;
                    u[i + 1] = v.y;
                }
            } else {
#pragma unroll
                for (int i = 0; i < LX; ++i) u[i] = __ldg(src + i);
            }
        } else {
#pragma unroll
            for (int i = 0; i < LX; ++i) u[i] = 0.0;
        }
        uint32_t hm = 0;  // largest high word of |u| in the pencil, then in the element
#pragma unroll
        for (int i = 0; i < LX; ++i) {
            umax_bits = max(umax_bits, (unsigned long long)__double_as_longlong(u[i]) & 0x7fffffffffffffffull);
            hm = max(hm, (uint32_t)__double2hiint(u[i]) & 0x7fffffffu);
        }
        if constexpr (C::ALIGNED) {  // the element's lanes of this warp first
            const unsigned seg_mask =
                (C::SEG == 32) ? 0xffffffffu : (((1u << C::SEG) - 1u) << (lane & ~(C::SEG - 1)));
            hm = __reduce_max_sync(seg_mask, hm);
            if ((lane & (C::SEG - 1)) == 0 && in_tile) atomicMax(&s_hx[lt], hm);
        } else if (in_tile) {
            atomicMax(&s_hx[lt], hm);
        }
        __syncthreads();
        const int kb = prescale_exponent(in_tile ? s_hx[lts] : 0u) << 20;
#pragma unroll
        for (int i = 0; i < LX; ++i) {
            if constexpr (DF) {
                d2f_split(u[i], kb, uh[i], ul[i]);
            } else {
                uh[i] = d2f_rz_scaled(u[i], kb);
                ul[i] = 0.0f;
            }
        }
    }

    // ---- forward transform in FP32 along i (registers), j, k (shared-memory
    // transposes).  In FP64 mode the FP32 coefficients settle every decision
    // they are provably on the right side of; the others are recomputed exactly.
    float ah[LX], al[LX];  // modal coefficients a[r][q=pa][p=pb], mode m = P + NP r
    if constexpr (DF && CUM) {  // the whole transform in float pairs
        f2 x[LX], y[LX];
#pragma unroll
        for (int i = 0; i < LX; ++i) x[i] = {uh[i], ul[i]};
        fwd1d_df<LX>(tab.Ah, tab.Al, x, y);
        if (in_tile) {
#pragma unroll
            for (int q = 0; q < LX; ++q) b1[pa * SX + pb * SY + q] = make_float2(y[q].h, y[q].l);
        }
        __syncthreads();
        if (in_tile) {
#pragma unroll
            for (int j = 0; j < LX; ++j) {
                const float2 v = b1[pa * SX + j * SY + pb];
                x[j] = {v.x, v.y};
            }
        }
        fwd1d_df<LX>(tab.Ah, tab.Al, x, y);
        if (in_tile) {
#pragma unroll
            for (int q = 0; q < LX; ++q) b2[pa * SX + q * SY + pb] = make_float2(y[q].h, y[q].l);
        }
        __syncthreads();
        if (in_tile) {
#pragma unroll
            for (int k = 0; k < LX; ++k) {
                const float2 v = b2[k * SX + pa * SY + pb];
                x[k] = {v.x, v.y};
            }
        }
        fwd1d_df<LX>(tab.Ah, tab.Al, x, y);
#pragma unroll
        for (int r = 0; r < LX; ++r) {
            ah[r] = y[r].h;
            al[r] = y[r].l;
        }
    } else {
        float x[LX], y[LX];
#pragma unroll
        for (int i = 0; i < LX; ++i) x[i] = uh[i];
        fwd1d<LX, float>(tab.Ah, x, y);
        if (in_tile) {
#pragma unroll
            for (int q = 0; q < LX; ++q) t1f[lts * C::BUFN + pa * SX + pb * SY + q] = y[q];
        }
        __syncthreads();
        if (in_tile) {
#pragma unroll
            for (int j = 0; j < LX; ++j) x[j] = t1f[lts * C::BUFN + pa * SX + j * SY + pb];
        }
        fwd1d<LX, float>(tab.Ah, x, y);
        if (in_tile) {
#pragma unroll
            for (int q = 0; q < LX; ++q) t2f[lts * C::BUFN + pa * SX + q * SY + pb] = y[q];
        }
        __syncthreads();
        if (in_tile) {
#pragma unroll
            for (int k = 0; k < LX; ++k) x[k] = t2f[lts * C::BUFN + k * SX + pa * SY + pb];
        }
        fwd1d<LX, float>(tab.Ah, x, y);
#pragma unroll
        for (int r = 0; r < LX; ++r) {
            ah[r] = y[r];
            al[r] = 0.0f;
        }
    }

    // ---- element energy and max |u|.  FP64 mode: S_e = sum w_i w_j w_k u^2
    // over the GLL points (Parseval's identity in nodal form), in float pairs
    // from the exact split of u.  FP32 mode: S_e = sum a^2 of the coefficients.
    f2 sp = {0.0f, 0.0f};
    if (active) {
        if constexpr (DF) {
#pragma unroll
            for (int i = 0; i < LX; ++i) {
                const float ph = uh[i] * uh[i];
                const float pl = fmaf(2.0f * uh[i], ul[i], fmaf(uh[i], uh[i], -ph));
                const float2 w = sWq[i * NP + P];
                df_fma_acc(sp, {w.x, w.y}, {ph, pl});
            }
            sp = df_norm(sp);
        } else {
#pragma unroll
            for (int r = 0; r < LX; ++r) sp.h = fmaf(ah[r], ah[r], sp.h);
        }
    }
    if constexpr (CUM) {  // cleared here, used after the barriers of the element reduction
        if constexpr (!DIRECT) {
            for (int i = tid; i < 64 * TILE; i += C::BLOCK) sbk[i] = 0ull;
        }
        if (tid < TILE) s_ncand[tid] = 0;
    }
    elem_reduce<LX, TILE_, DF>(red, selem, sp, umax_bits, true, 0, 2, n_here);  // S' -> [0], max|u| -> [2]

    // ---- per element (one thread each): t = tau S, step s, magnitude threshold g
    if (tid < TILE) {
        const int l = tid;
        const double Se = selem[l * 8 + 0];
        int step = INT16_MIN, mode = 0;  // 0: keep none, 1: threshold, 2: keep all (lossless)
        double g = 0.0;
        if constexpr (CUM) {
            s_cK[l] = 0;
            s_tint[l] = 0ull;
        }
        const uint32_t hx = s_hx[l];
        const int ke = prescale_exponent(hx);
        if (l < n_here) {
            if (!isfinite(Se) || hmax_bad(hx)) {
                atomicOr(&ctl->status, (unsigned)SEMR_STATUS_NONFINITE);
            } else if (p.lossless) {
                mode = 2;
                if (hmax_tiny(hx)) atomicOr(&ctl->status, (unsigned)SEMR_STATUS_TINY);
            } else if (hmax_tiny(hx)) {  // zeros and subnormals only: keeps nothing, norms 0
                if (hx != 0u) atomicOr(&ctl->status, (unsigned)SEMR_STATUS_TINY);
            } else {
                // t' = tau S' of the prescaled block (S' >= min w_i w_j w_k > 3e-6 and tau > 2^-60:
                // normal); the element's t = t' 2^2ke, so ex = ex' + 2 ke and s_e = s' + ke with
                // s' = floor((ex' - 1) / 2).  s_step holds s', which the codes and the
                // reconstruction use; the payload gets s' + ke
                const double t = p.tau * Se;
                const long long bits = __double_as_longlong(t);
                const int exs = (int)((bits >> 52) & 0x7ff) - 1022;
                const int ex = exs + 2 * ke;
                if (!isfinite(t) || !(t >= DBL_MIN) || ex > 1024) {  // t overflows FP64
                    atomicOr(&ctl->status, (unsigned)SEMR_STATUS_NONFINITE);
                } else if (ex >= -1021) {  // t >= 2^-1022, the smallest normal double
                    const int st = (exs - 1) >> 1;
                    if (st >= -250 && st <= 250) {  // 2^-s' as a product of two normal floats
                        step = st;
                        mode = 1;
                        if constexpr (CUM) {  // t' in [2^(ex'-1), 2^ex'): K = 48 - ex', floor(t' 2^K) = M >> 5
                            s_cK[l] = 48 - exs;
                            s_tint[l] = (((unsigned long long)bits & 0xfffffffffffffull) | (1ull << 52)) >> 5;
                        }
                        // FP64 mode refines g to the exact double threshold only for elements
                        // with coefficients it recomputes; the float threshold settles the rest
                        g = (double)threshold_abs32_fast(t);
                    } else {
                        atomicOr(&ctl->status, (unsigned)SEMR_STATUS_NONFINITE);
                    }
                }
            }
        }
        const f2 gp = df_from_double(g);  // FP32 mode: g is a float, the low word is 0
        s_g[2 * l] = gp.h;
        s_g[2 * l + 1] = gp.l;
        s_step[l] = step;
        s_mode[l] = mode;
        // bound on |a_fp32 - a|: (H + 2) roundings per folded contraction (H terms, the fold,
        // the table), 3 contractions, 2 more for the input split; (|A|^3 |u|)_m <= 2^1.5 max|u|
        // because every row of A has sum |A_pi| <= sqrt(2); a factor 2 of safety on top.
        // max |u 2^-ke| rounded toward zero (the top 20 mantissa bits of hx, in [1, 2)).
        constexpr float kMarg = (3.0f * ((LX + 1) / 2 + 2) + 2.0f) * 5.9604645e-8f * 2.8285f * 2.0f;
        const float umx = hmax_tiny(hx) ? 0.0f : __uint_as_float(0x3f800000u | ((hx & 0xfffffu) << 3));
        s_marg[l] = kMarg * umx * 1.000002f;
    }
    __syncthreads();
    const int emode = in_tile ? s_mode[lt] : 0;
    const int step = (in_tile && emode == 1) ? s_step[lt] : 0;
    f2 g2 = in_tile ? f2{s_g[2 * lt], s_g[2 * lt + 1]} : f2{0.0f, 0.0f};

    if constexpr (DF && !CUM) {
        // ---- decisions the FP32 coefficients cannot settle: recompute them exactly
        const int sdn1 = (-step) >> 1, sdn2 = -step - sdn1;
        const float sc = pow2f(sdn1) * pow2f(sdn2);  // 2^-s, exact
        uint32_t amb = 0;
        if (active && emode == 1) {
            const float Mg = s_marg[lt] + g2.h * 2.4e-7f;  // plus the float rounding of g +- M
            const float Mq = Mg * sc;
#pragma unroll
            for (int r = 0; r < LX; ++r) {
                const float aa = fabsf(ah[r]);
                if (aa >= g2.h + Mg) {  // surely kept: is the rounding decision sure too?
                    const float y = aa * sc;
                    if (fabsf((y - floorf(y)) - 0.5f) <= Mq + y * 1.2e-7f) amb |= 1u << r;
                } else if (!(aa < g2.h - Mg)) {
                    amb |= 1u << r;  // too close to the threshold
                }
            }
        }
        for (int round = 0;; ++round) {  // rounds of up to AMB_CAP entries per tile
            if (tid == 0) s_namb[0] = 0;
            if (tid < TILE) s_namb[1 + tid] = 0;
            __syncthreads();
            if (amb) s_namb[1 + lt] = 1;
            int ent[LX];
#pragma unroll
            for (int r = 0; r < LX; ++r) {
                ent[r] = -1;
                if (amb & (1u << r)) {
                    const int k = atomicAdd(&s_namb[0], 1);
                    if (k < AMB_CAP) {
                        s_amb[k] = (lt << 16) | (P + NP * r);
                        ent[r] = k;
                    }
                }
            }
            __syncthreads();
            const int total = s_namb[0];
            if (total == 0) break;
            if (tid == 0) atomicAdd(&ctl->recomputed, (unsigned)(total < AMB_CAP ? total : AMB_CAP));
            if (tid < TILE && s_namb[1 + tid] && s_mode[tid] == 1) {  // exact double threshold of the element
                const f2 ge = df_from_double(threshold_abs64(p.tau * selem[tid * 8 + 0]));
                s_g[2 * tid] = ge.h;
                s_g[2 * tid + 1] = ge.l;
            }
            // Each entry in hardware FP64 from the element's doubles (reread from global memory,
            // where L2 still holds them): a kept coefficient can be as small as ~7e-6 max|u| at
            // tau = 1e-6 in a spiky element, where float pairs would carry a relative error near
            // the 1e-9 band of the decisions.  Rare, so the slow FP64 pipe costs little.
            const int n_amb = total < AMB_CAP ? total : AMB_CAP;
            for (int k = 0; k < n_amb; ++k) {
                const int code = s_amb[k];
                const int el = code >> 16, m = code & 0xffff;
                double c = 0.0;
                if (lt == el && active) {
                    const int pp = m % LX, qq = (m / LX) % LX, rr = m / NP;
                    const double* src = p.fields[f] + e * N3 + P * LX;
                    double xs = 0.0;
#pragma unroll
                    for (int i = 0; i < LX; ++i) xs = fma(tab.A64[pp * LX + i], __ldg(src + i), xs);
                    c = (xs * tab.A64[qq * LX + pb]) * tab.A64[rr * LX + pa];
                }
                // CTA-wide sum (only element el contributes), in a fixed order
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                if (lane == 0) reinterpret_cast<double*>(red)[tid >> 5] = c;
                __syncthreads();
                if (tid == 0) {
                    double a = 0.0;
                    for (int w = 0; w < C::NW; ++w) a += reinterpret_cast<double*>(red)[w];
                    const f2 ap = df_from_double(a * pow2d(-prescale_exponent(s_hx[el])));  // u 2^-ke
                    s_ambv[2 * k] = ap.h;
                    s_ambv[2 * k + 1] = ap.l;
                }
                __syncthreads();
            }
#pragma unroll
            for (int r = 0; r < LX; ++r) {
                if (ent[r] >= 0) {  // exact coefficient replaces the FP32 one
                    ah[r] = s_ambv[2 * ent[r]];
                    al[r] = s_ambv[2 * ent[r] + 1];
                    amb &= ~(1u << r);
                }
            }
            if (total <= AMB_CAP) break;
            __syncthreads();
        }
        if (in_tile) g2 = f2{s_g[2 * lt], s_g[2 * lt + 1]};  // exact where it was refined
    }

    // ---- cumulative variant: the boundary key T of each element
    constexpr unsigned long long KCLAMP = 1ull << 50;  // key of every energy >= 2t: always kept
    const int cK = (CUM && in_tile) ? s_cK[lt] : 0;
    auto energy_key = [&](int r) -> unsigned long long {  // floor(a^2 2^K) from the exact square
        const f2 e2 = df_mul({ah[r], al[r]}, {ah[r], al[r]});
        const long long v = (long long)fixp(e2.h, cK) + fixp_signed(e2.l, cK);
        if (v <= 0) return 0ull;
        return ((unsigned long long)v >= (1ull << 49)) ? KCLAMP : (unsigned long long)v;
    };
    unsigned long long sT = ~0ull;
    unsigned long long ek[CUM ? LX : 1];  // energy keys of the pencil's coefficients (0 when not selecting)
    if constexpr (CUM) {
        const int wid = tid >> 5;
        const bool sel = active && emode == 1;
#pragma unroll
        for (int r = 0; r < LX; ++r) ek[r] = sel ? energy_key(r) : 0ull;
        if constexpr (DIRECT) {
            if (sel) {
#pragma unroll
                for (int r = 0; r < LX; ++r) scand[lt * N3 + P + NP * r] = ek[r];
            }
        } else {
            if (sel) {
#pragma unroll
                for (int r = 0; r < LX; ++r) {
                    if (ek[r]) atomicAdd(&sbk[lt * 64 + (64 - __clzll((long long)ek[r]))], ek[r]);
                }
            }
            __syncthreads();
            for (int l = wid; l < TILE; l += C::NW) {  // octave of T: first prefix of octave sums above t
                const unsigned long long lo = sbk[l * 64 + lane], hi = sbk[l * 64 + 32 + lane];
                const unsigned long long ilo = warp_incl_scan_u64(lo), ihi = warp_incl_scan_u64(hi);
                const unsigned long long tot = __shfl_sync(0xffffffffu, ilo, 31);
                const unsigned long long tt = s_tint[l];
                const bool ok = l < n_here && s_mode[l] == 1;
                const unsigned m1 = __ballot_sync(0xffffffffu, ok && ilo > tt);
                const unsigned m2 = __ballot_sync(0xffffffffu, ok && tot + ihi > tt);
                int bs = -1;
                unsigned long long base = 0ull;
                if (m1) {
                    bs = __ffs(m1) - 1;
                    base = __shfl_sync(0xffffffffu, ilo - lo, bs);
                } else if (m2) {
                    const int j = __ffs(m2) - 1;
                    bs = 32 + j;
                    base = tot + __shfl_sync(0xffffffffu, ihi - hi, j);
                }
                if (lane == 0) {
                    s_bstar[l] = bs;
                    s_base[l] = base;
                }
            }
            __syncthreads();
            const int bs = in_tile ? s_bstar[lt] : -1;
            if (sel && bs > 0) {  // gather the keys of that octave
#pragma unroll
                for (int r = 0; r < LX; ++r) {
                    if (ek[r] && (64 - __clzll((long long)ek[r])) == bs)
                        scand[lt * N3 + atomicAdd(&s_ncand[lt], 1)] = ek[r];
                }
            }
        }
        __syncthreads();
        for (int l = wid; l < TILE; l += C::NW) {  // one warp per element: T from the octave's keys
            unsigned long long T = ~0ull;
            const bool ok = l < n_here && s_mode[l] == 1 && (DIRECT || s_bstar[l] > 0);
            if (ok) {
                const int c = DIRECT ? N3 : s_ncand[l];
                const unsigned long long base = DIRECT ? 0ull : s_base[l];
                const unsigned long long tt = s_tint[l];
                const unsigned long long* cand = scand + (size_t)l * N3;
                if (c <= 32) {  // sort, scan, first inclusive sum above the budget
                    unsigned long long v = (lane < c) ? cand[lane] : ~0ull;
                    v = warp_sort_u64(v);
                    const unsigned long long inc = warp_incl_scan_u64(lane < c ? v : 0ull);
                    const unsigned m = __ballot_sync(0xffffffffu, lane < c && base + inc > tt);
                    if (m) T = __shfl_sync(0xffffffffu, v, __ffs(m) - 1);
                } else {  // bisection on the key value: smallest v with base + sum(keys <= v) > t
                    const int bs = DIRECT ? 1 : s_bstar[l];
                    unsigned long long lo = 1ull << (bs - 1), hi = (bs > 50) ? KCLAMP : (1ull << bs) - 1ull;
                    while (lo < hi) {
                        const unsigned long long mid = lo + (hi - lo) / 2;
                        unsigned long long sm = 0ull;
                        for (int i = lane; i < c; i += 32) {
                            const unsigned long long k = cand[i];
                            if (k <= mid) sm += k;
                        }
                        sm = warp_sum_u62(sm);
                        if (base + sm > tt) hi = mid;
                        else lo = mid + 1;
                    }
                    T = lo;
                }
            }
            if (lane == 0) s_T[l] = T;
        }
        __syncthreads();
        if (in_tile) sT = s_T[lt];
    }

    // ---- mask bits: ballots when elements are whole warps, else shared atomics
    uint32_t keepbits = 0;
    uint32_t bw[LX];  // ballot word of mode P + NP r (ballot path)
#pragma unroll
    for (int r = 0; r < LX; ++r) {
        bool k;
        if constexpr (CUM) k = ek[r] >= sT;
        else if constexpr (DF) k = df_ge(df_abs({ah[r], al[r]}), g2);
        else k = fabsf(ah[r]) >= g2.h;
        k = active && (emode == 2 || (emode == 1 && k));
        keepbits |= (k ? 1u : 0u) << r;
        if constexpr (C::BALLOT) {
            bw[r] = __ballot_sync(0xffffffffu, k);
            if (lane == 0 && in_tile) smask[lt * MW + (P >> 5) + (NP / 32) * r] = bw[r];
        } else {
            bw[r] = 0;
            if (k) {
                const int m = P + NP * r;
                atomicOr(&smask[lt * MW + (m >> 5)], 1u << (m & 31));
            }
        }
    }
    __syncthreads();
    {  // word prefix popcounts and counts, one warp per element
        const int warp = tid >> 5;
        for (int l = warp; l < TILE; l += C::NW) {
            uint32_t carry = 0;
            for (int w0 = 0; w0 < MW; w0 += 32) {
                const int w = w0 + lane;
                const uint32_t c = (w < MW && l < n_here) ? __popc(smask[l * MW + w]) : 0u;
                uint32_t incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                if (w < MW) swpre[l * MW + w] = carry + incl - c;
                carry += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (lane == 0) s_cnt[l] = (int)carry;
        }
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0, big = 0;
        for (int l = 0; l < TILE; ++l) {
            s_epre[l] = acc;
            const int c = (l < n_here) ? s_cnt[l] : 0;
            acc += c;
            big |= (c > SPARSE_MAX) || (l < n_here && s_mode[l] == 2);
        }
        s_epre[TILE] = acc;
        s_flag[0] = big;
        if (tok) st_release_u64(&tile_state[tile], (tile == 0 ? kFlagPrefix : kFlagAggregate) | ((uint64_t)acc & kValueMask));
    }
    __syncthreads();
    const bool dense = s_flag[0] != 0;

    // ---- quantise: y = a 2^-s (exact, two float factors), code = rint(y), ties to even
    const int sd1 = (-step) >> 1, sd2 = -step - sd1;  // 2^-s = 2^sd1 2^sd2
    const float qd1 = pow2f(sd1), qd2 = pow2f(sd2);
    const int su1 = step >> 1, su2 = step - su1;      // 2^s = 2^su1 2^su2
    const float qu1 = pow2f(su1), qu2 = pow2f(su2);
    float ch[LX];  // code values (exact floats), 0 when dropped; lossless: the coefficient (hi)
    if (emode == 2) {
        // lossless mode: every mode kept, raw FP64 coefficients stored
#pragma unroll
        for (int r = 0; r < LX; ++r) {
            ch[r] = ah[r];
            if (keepbits & (1u << r)) {
                const int m = P + NP * r;
                const int rank = (int)swpre[lt * MW + (m >> 5)] +
                                 __popc(smask[lt * MW + (m >> 5)] & ((1u << (m & 31)) - 1u));
                if constexpr (S::code_b == 8)  // the launcher sends lossless work only to kernels with 8-B staging
                    reinterpret_cast<double*>(scodes)[s_epre[lt] + rank] =
                        ((double)ah[r] + (double)al[r]) * pow2d(prescale_exponent(s_hx[lt]));
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < LX; ++r) {
            ch[r] = 0.0f;
            if constexpr (C::BALLOT) {
                if (bw[r] == 0u) continue;  // warp-uniform: no lane keeps mode r
            }
            const bool k = keepbits & (1u << r);
            if (k) {
                const float yh = (ah[r] * qd1) * qd2;
                float c;
                if (width == 2) {
                    c = (yh + 12582912.0f) - 12582912.0f;  // round half to even, exact for |y| < 2^22
                } else {
                    c = rintf(yh);
                }
                if constexpr (DF) {  // correct by the low word: rounds the pair yh + yl
                    const float diff = (yh - c) + (al[r] * qd1) * qd2;
                    c += (diff > 0.5f) ? 1.0f : ((diff < -0.5f) ? -1.0f : 0.0f);
                }
                ch[r] = c;
                const int m = P + NP * r;
                const uint32_t wm = C::BALLOT ? bw[r] : smask[lt * MW + (m >> 5)];
                const int rank = (int)swpre[lt * MW + (m >> 5)] + __popc(wm & ((1u << (m & 31)) - 1u));
                const int pos = s_epre[lt] + rank;
                if (width == 2) reinterpret_cast<int16_t*>(scodes)[pos] = (int16_t)(int)c;
                else reinterpret_cast<int32_t*>(scodes)[pos] = (int32_t)c;
                if (rank < KL) {  // only read while every element keeps at most SPARSE_MAX <= KL modes
                    skm[lt * KL + rank] = (uint16_t)m;
                    skc[lt * KL + rank] = c;
                }
            }
        }
    }
    __syncthreads();

    // ---- reconstruction u~ of the pencil (k=pa, j=pb), as pairs in FP64 mode
    float vh[LX], vl[LX];
#pragma unroll
    for (int i = 0; i < LX; ++i) {
        vh[i] = 0.0f;
        vl[i] = 0.0f;
    }
    if (!dense) {
        if (active) {
            const int nk = s_cnt[lt];
            const int rowj = pb * PT, rowk = pa * PT;
            for (int t = 0; t < nk; ++t) {
                const int m = skm[lt * KL + t];
                const float cs = (skc[lt * KL + t] * qu1) * qu2;  // c 2^s, exact
                const int pp = m % LX, qq = (m / LX) % LX, rr = m / NP;
                float ch_[LX], cl_[LX];  // column p of Phi: Phi[i][pp], i = 0..LX-1
                if constexpr (LX % 4 == 0) {
#pragma unroll
                    for (int i = 0; i < LX; i += 4) {
                        const float4 h4 = *reinterpret_cast<const float4*>(sPTh + pp * CS + i);
                        ch_[i] = h4.x; ch_[i + 1] = h4.y; ch_[i + 2] = h4.z; ch_[i + 3] = h4.w;
                        if constexpr (DF) {
                            const float4 l4 = *reinterpret_cast<const float4*>(sPTl + pp * CS + i);
                            cl_[i] = l4.x; cl_[i + 1] = l4.y; cl_[i + 2] = l4.z; cl_[i + 3] = l4.w;
                        }
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < LX; ++i) {
                        ch_[i] = sPTh[pp * CS + i];
                        if constexpr (DF) cl_[i] = sPTl[pp * CS + i];
                    }
                }
                if constexpr (DF) {
                    const f2 b = df_mulf(df_mul({sPh[rowj + qq], sPl[rowj + qq]}, {sPh[rowk + rr], sPl[rowk + rr]}), cs);
#pragma unroll
                    for (int i = 0; i < LX; ++i) {  // renormalised once after the loop
                        f2 acc = {vh[i], vl[i]};
                        df_fma_acc(acc, b, {ch_[i], cl_[i]});
                        vh[i] = acc.h;
                        vl[i] = acc.l;
                    }
                } else {
                    const float b = cs * sPh[rowj + qq] * sPh[rowk + rr];
#pragma unroll
                    for (int i = 0; i < LX; ++i) vh[i] = fmaf(b, ch_[i], vh[i]);
                }
            }
            if constexpr (DF) {
#pragma unroll
                for (int i = 0; i < LX; ++i) {
                    const f2 n = df_norm({vh[i], vl[i]});
                    vh[i] = n.h;
                    vl[i] = n.l;
                }
            }
        }
    } else {
        // dense folded inverse: along r (registers), q, p (shared-memory transposes)
        if constexpr (DF) {
            f2 x[LX], y[LX];
#pragma unroll
            for (int r = 0; r < LX; ++r) x[r] = (emode == 2) ? f2{ah[r], al[r]} : f2{(ch[r] * qu1) * qu2, 0.0f};
            inv1d_df<LX>(tab.Ph, tab.Pl, x, y);  // y[k] = v[k][q=pa][p=pb]
            if (in_tile) {
#pragma unroll
                for (int k = 0; k < LX; ++k) b1[k * SX + pa * SY + pb] = make_float2(y[k].h, y[k].l);
            }
            __syncthreads();
            if (in_tile) {
#pragma unroll
                for (int q = 0; q < LX; ++q) {
                    const float2 v = b1[pa * SX + q * SY + pb];
                    x[q] = {v.x, v.y};
                }
            }
            inv1d_df<LX>(tab.Ph, tab.Pl, x, y);  // y[j] = v2[k=pa][j][p=pb]
            if (in_tile) {
#pragma unroll
                for (int j = 0; j < LX; ++j) b2[pa * SX + j * SY + pb] = make_float2(y[j].h, y[j].l);
            }
            __syncthreads();
            if (in_tile) {
#pragma unroll
                for (int q = 0; q < LX; ++q) {
                    const float2 v = b2[pa * SX + pb * SY + q];
                    x[q] = {v.x, v.y};
                }
            }
            inv1d_df<LX>(tab.Ph, tab.Pl, x, y);
#pragma unroll
            for (int i = 0; i < LX; ++i) {
                vh[i] = y[i].h;
                vl[i] = y[i].l;
            }
        } else {
            float x[LX], y[LX];
#pragma unroll
            for (int r = 0; r < LX; ++r) x[r] = (emode == 2) ? ch[r] : (ch[r] * qu1) * qu2;
            inv1d<LX, float>(tab.Ph, x, y);
            if (in_tile) {
#pragma unroll
                for (int k = 0; k < LX; ++k) b1[k * SX + pa * SY + pb] = y[k];
            }
            __syncthreads();
            if (in_tile) {
#pragma unroll
                for (int q = 0; q < LX; ++q) x[q] = b1[pa * SX + q * SY + pb];
            }
            inv1d<LX, float>(tab.Ph, x, y);
            if (in_tile) {
#pragma unroll
                for (int j = 0; j < LX; ++j) b2[pa * SX + j * SY + pb] = y[j];
            }
            __syncthreads();
            if (in_tile) {
#pragma unroll
                for (int q = 0; q < LX; ++q) x[q] = b2[pa * SX + pb * SY + q];
            }
            inv1d<LX, float>(tab.Ph, x, y);
#pragma unroll
            for (int i = 0; i < LX; ++i) vh[i] = y[i];
        }
    }

    // ---- errors of the pencil: e2 = sum w (u - u~)^2 (without J), Linf = max |u - u~|
    f2 e2p = {0.0f, 0.0f};
    unsigned long long linf_bits = 0;
    if (active) {
        if constexpr (DF) {
            f2 dmax = {0.0f, 0.0f};
#pragma unroll
            for (int i = 0; i < LX; ++i) {
                const f2 d = df_sub({uh[i], ul[i]}, {vh[i], vl[i]});
                const float2 w = sWq[i * NP + P];
                df_fma_acc(e2p, df_mul({w.x, w.y}, d), d);
                const f2 ad = df_abs(d);
                if (df_ge(ad, dmax)) dmax = ad;
            }
            e2p = df_norm(e2p);
            linf_bits = pair_to_double_bits(dmax);
        } else {
            unsigned dm = 0;
#pragma unroll
            for (int i = 0; i < LX; ++i) {
                const float d = uh[i] - vh[i];
                e2p.h = fmaf(wq32[i] * d, d, e2p.h);
                dm = max(dm, __float_as_uint(fabsf(d)));
            }
            linf_bits = dm;
        }
        if (p.write_recon && p.recon[f] && tok) {  // u~ = u~' 2^ke (exact)
            double* dst = p.recon[f] + e * N3 + P * LX;
            const double sc = pow2d(prescale_exponent(s_hx[lt]));
#pragma unroll
            for (int i = 0; i < LX; ++i) dst[i] = ((double)vh[i] + (double)vl[i]) * sc;
        }
    }
    elem_reduce<LX, TILE_, DF>(red, selem, e2p, linf_bits, DF, 1, 3, n_here);  // e2/J -> [1], Linf -> [3]

    // ---- look-back (one warp) and tile partials
    if (tid < 32) {
        const uint64_t ex = lookback_warp(tile_state, tile, (uint64_t)s_epre[TILE], &ctl->status);
        if (tid == 0) s_tile[1] = ex;
    }
    if (tid == 32 % C::BLOCK && tok) {  // another warp, when there is one
        double s0 = 0.0, s1 = 0.0, m2 = 0.0, m3 = 0.0;
        for (int l = 0; l < n_here; ++l) {  // back from the prescaled block: 2^2ke, 2^ke
            const double J = p.jac[e0 + l];
            const double sc = pow2d(prescale_exponent(s_hx[l]));
            s0 += J * ((selem[l * 8 + 1] * sc) * sc);
            s1 += J * ((selem[l * 8 + 0] * sc) * sc);
            m2 = fmax(m2, selem[l * 8 + 3] * sc);
            m3 = fmax(m3, selem[l * 8 + 2]);
        }
        double* tp = tile_part + 4 * tile;
        tp[0] = s0;
        tp[1] = s1;
        tp[2] = m2;
        tp[3] = m3;
    }
    __syncthreads();
    const uint64_t tile_excl = s_tile[1];

    // ---- writes: codes (contiguous for the tile), masks, steps, counts, element report
    {
        const uint64_t ncodes = (uint64_t)s_epre[TILE];
        const uint64_t gbyte = p.code_base + (uint64_t)width * tile_excl;
        const uint64_t nbytes = (uint64_t)width * ncodes;
        if (!tok) {
            // (bounds build) nothing of this tile is written
        } else if (gbyte + nbytes <= p.payload_cap) {
            uint8_t* dst = p.payload + gbyte;
            if (width == 8) {
                if constexpr (S::code_b == 8) {
                    const double* sc = reinterpret_cast<const double*>(scodes);
                    for (uint64_t i = tid; i < ncodes; i += C::BLOCK) reinterpret_cast<double*>(dst)[i] = sc[i];
                }
            } else if (width == 4) {
                const int32_t* sc = reinterpret_cast<const int32_t*>(scodes);
                for (uint64_t i = tid; i < ncodes; i += C::BLOCK) reinterpret_cast<int32_t*>(dst)[i] = sc[i];
            } else {
                const int16_t* sc = reinterpret_cast<const int16_t*>(scodes);
                for (uint64_t i = tid; i < ncodes; i += C::BLOCK) reinterpret_cast<int16_t*>(dst)[i] = sc[i];
            }
        } else if (tid == 0 && nbytes > 0) {
            atomicOr(&ctl->status, (unsigned)SEMR_STATUS_OVERFLOW);
        }
    }
    if (tok) {
        constexpr int mb = (N3 + 7) / 8;
        uint8_t* fsec = p.payload + p.header_bytes + (uint64_t)f * p.fixed_bytes;
        if constexpr ((mb % 4) == 0) {  // whole words: element masks are word-aligned
            uint32_t* mdst = reinterpret_cast<uint32_t*>(fsec) + (uint64_t)e0 * (mb / 4);
            for (int i = tid; i < n_here * (mb / 4); i += C::BLOCK) mdst[i] = smask[(i / (mb / 4)) * MW + i % (mb / 4)];
        } else {
            uint8_t* mdst = fsec + (uint64_t)e0 * mb;
            const uint8_t* msrc = reinterpret_cast<const uint8_t*>(smask);
            for (int i = tid; i < n_here * mb; i += C::BLOCK) {
                const int l = i / mb, b = i % mb;
                mdst[i] = msrc[l * MW * 4 + b];
            }
        }
        int16_t* sdst = reinterpret_cast<int16_t*>(fsec + pad16((uint64_t)p.n_elem * mb));
        uint16_t* cdst = reinterpret_cast<uint16_t*>(fsec + pad16((uint64_t)p.n_elem * mb) + pad16(2ull * p.n_elem));
        if (tid < n_here) {
            sdst[e0 + tid] = (int16_t)(s_mode[tid] == 1 ? s_step[tid] + prescale_exponent(s_hx[tid]) : INT16_MIN);
            cdst[e0 + tid] = (uint16_t)s_cnt[tid];
        }
        if (e0 + n_here == p.n_elem && tid < 16) {
            const uint64_t me = (uint64_t)p.n_elem * mb;
            if (me + tid < pad16(me)) fsec[me + tid] = 0;
            const uint64_t se = 2ull * p.n_elem;
            uint8_t* sb = reinterpret_cast<uint8_t*>(sdst);
            uint8_t* cb = reinterpret_cast<uint8_t*>(cdst);
            if (se + tid < pad16(se)) {
                sb[se + tid] = 0;
                cb[se + tid] = 0;
            }
        }
        if (p.elem_report && tid < 3 * n_here) {
            const int l = tid / 3, c = tid % 3;
            const double J = p.jac[e0 + l];
            const double sc = pow2d(prescale_exponent(s_hx[l]));
            const double v = (c == 0) ? J * ((selem[l * 8 + 1] * sc) * sc)
                                      : (c == 1) ? J * ((selem[l * 8 + 0] * sc) * sc) : selem[l * 8 + 3] * sc;
            p.elem_report[((uint64_t)f * p.n_elem + e0) * 3 + tid] = v;
        }
    }
    __syncthreads();  // shared state is reused by the next tile
    }
}

}  // namespace semr

// ------------------------------------------------------------ launcher

namespace semr {
namespace {

template <int LX>
FastTables<LX> make_tables() {
    FastTables<LX> tab;
    double A[LX * LX], Phi[LX * LX], w[LX];
    basis_tables(LX, A, Phi, w);
    for (int i = 0; i < LX * LX; ++i) {
        tab.A64[i] = A[i];
        tab.Ah[i] = (float)A[i];
        tab.Al[i] = (float)(A[i] - (double)tab.Ah[i]);
        tab.Ph[i] = (float)Phi[i];
        tab.Pl[i] = (float)(Phi[i] - (double)tab.Ph[i]);
    }
    for (int i = 0; i < LX; ++i) {
        tab.wh[i] = (float)w[i];
        tab.wl[i] = (float)(w[i] - (double)tab.wh[i]);
    }
    return tab;
}

// Persistent grid: as many CTAs as fit on the GPU at once, never more than tiles.
template <typename K>
int persistent_grid(K kernel, int block, size_t smem, uint64_t tiles, unsigned* grid) {
    cudaError_t err;
    int dev = 0, sms = 0, per_sm = 0;
    if ((err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return (int)err;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return (int)err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem)) != cudaSuccess)
        return (int)err;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    *grid = (unsigned)std::min<uint64_t>(tiles, (uint64_t)sms * per_sm);
    return 0;
}

template <int LX, int MODE, int TILE_>
int launch_fast_single(const LaunchParams& p, void* stream) {
    using C = FCfg<LX, TILE_>;
    const FastTables<LX> tab = make_tables<LX>();
    const size_t smem = FSmem<LX, MODE, TILE_>::bytes;
    unsigned grid = 0;
    const uint64_t tiles = (uint64_t)p.n_fields * p.tiles_per_field;
    int rc = persistent_grid(reduce_fast_kernel<LX, MODE, TILE_, false>, C::BLOCK, smem, tiles, &grid);
    if (rc) return rc;
    BatchQueue q{};
    reduce_fast_kernel<LX, MODE, TILE_, false><<<grid, C::BLOCK, smem, (cudaStream_t)stream>>>(p, q, tab);
    return (int)cudaGetLastError();
}

template <int LX, int MODE, int TILE_>
int launch_fast_batch(const BatchQueue& q, void* stream) {
    using C = FCfg<LX, TILE_>;
    const FastTables<LX> tab = make_tables<LX>();
    const size_t smem = FSmem<LX, MODE, TILE_>::bytes;
    unsigned grid = 0;
    int rc = persistent_grid(reduce_fast_kernel<LX, MODE, TILE_, true>, C::BLOCK, smem, q.total_tiles, &grid);
    if (rc) return rc;
    LaunchParams p0{};
    reduce_fast_kernel<LX, MODE, TILE_, true><<<grid, C::BLOCK, smem, (cudaStream_t)stream>>>(p0, q, tab);
    return (int)cudaGetLastError();
}

template <int MODE>
int single_mode(const LaunchParams& p, int lx, void* stream) {
    switch (lx) {
        case 2: return launch_fast_single<2, MODE, tile_elems(2)>(p, stream);
        case 3: return launch_fast_single<3, MODE, tile_elems(3)>(p, stream);
        case 4: return launch_fast_single<4, MODE, tile_elems(4)>(p, stream);
        case 5: return launch_fast_single<5, MODE, tile_elems(5)>(p, stream);
        case 6: return launch_fast_single<6, MODE, tile_elems(6)>(p, stream);
        case 7: return launch_fast_single<7, MODE, tile_elems(7)>(p, stream);
        case 8: return launch_fast_single<8, MODE, tile_elems(8)>(p, stream);
        case 9: return launch_fast_single<9, MODE, tile_elems(9)>(p, stream);
        case 10: return launch_fast_single<10, MODE, tile_elems(10)>(p, stream);
        case 11: return launch_fast_single<11, MODE, tile_elems(11)>(p, stream);
        case 12: return launch_fast_single<12, MODE, tile_elems(12)>(p, stream);
        default: return (int)cudaErrorInvalidValue;
    }
}

// Batched launches: every lx with its default tile; lx 6, 8, 10 with a second
// tile size the autotuner may pick.
template <int MODE>
int batch_mode(const BatchQueue& q, int lx, int tile, void* stream) {
#define SEMR_BATCH_CASE(L, T) \
    if (lx == L && tile == T) return launch_fast_batch<L, MODE, T>(q, stream);
    SEMR_BATCH_CASE(2, tile_elems(2))
    SEMR_BATCH_CASE(3, tile_elems(3))
    SEMR_BATCH_CASE(4, tile_elems(4))
    SEMR_BATCH_CASE(5, tile_elems(5))
    SEMR_BATCH_CASE(6, tile_elems(6))
    SEMR_BATCH_CASE(6, 16)
    SEMR_BATCH_CASE(7, tile_elems(7))
    SEMR_BATCH_CASE(8, tile_elems(8))
    SEMR_BATCH_CASE(8, 8)
    SEMR_BATCH_CASE(9, tile_elems(9))
    SEMR_BATCH_CASE(10, tile_elems(10))
    SEMR_BATCH_CASE(10, 4)
    SEMR_BATCH_CASE(11, tile_elems(11))
    SEMR_BATCH_CASE(12, tile_elems(12))
#undef SEMR_BATCH_CASE
    return (int)cudaErrorInvalidValue;
}

}  // namespace

int tile_variants(int lx, int* out, int cap) {
    int v[2] = {tile_elems(lx), 0};
    int n = 1;
    if (lx == 6) v[n++] = 16;
    if (lx == 8) v[n++] = 8;
    if (lx == 10) v[n++] = 4;
    for (int i = 0; i < n && i < cap; ++i) out[i] = v[i];
    return n;
}

int launch_reduce_fast(const LaunchParams& p, int lx, void* stream) {
    // lossless FP64 (8-byte raw coefficients) belongs to the hardware-FP64 kernel
    if (p.lossless && p.precision != SEMR_FP32) return (int)cudaErrorInvalidValue;
    if (p.cumulative)
        return p.precision == SEMR_FP32 ? single_mode<MODE_F32 | MODE_CUM>(p, lx, stream)
                                        : single_mode<MODE_DF64 | MODE_CUM>(p, lx, stream);
    return p.precision == SEMR_FP32 ? single_mode<MODE_F32>(p, lx, stream) : single_mode<MODE_DF64>(p, lx, stream);
}

int launch_reduce_fast_batch(const BatchQueue& q, int lx, int precision, int tile, void* stream) {
    // items are validated on the host: FP64 lossless items are refused when the batch is created
    return precision == SEMR_FP32 ? batch_mode<MODE_F32>(q, lx, tile, stream)
                                  : batch_mode<MODE_DF64>(q, lx, tile, stream);
}

}  // namespace semr
